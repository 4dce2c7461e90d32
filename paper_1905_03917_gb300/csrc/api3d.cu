// api3d.cu -- host context of the three-dimensional solver (include/sif3d.h):
// memory, the interaction step, the single-time-step step and the
// accelerated cycle of Sec. 3.1 issued from the host on the context's
// stream.  The cycle's decisions (time steps, the role of each fluid, the
// last sub-step) are taken on the host from maxima reduced on the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sif3d.h"
#include "sif3d_internal.cuh"

unsigned long long k3_fv_launches();

struct sif3_ctx {
  sif3_config cfg;
  Grid3 g;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  char *pool = nullptr;
  size_t pool_bytes = 0;
  double *q[2][S3_NC], *w[2][S3_NC], *q0[2][S3_NC];
  double *prev[S3_NC], *fut[S3_NC], *qi[S3_NC];
  double *xc[4], *xn[4], *xp[4], *ul[3];
  double *phi, *phi0, *lphi, *p0, *old, *alpha, *ax, *ay, *az, *sx, *sy, *sz, *corner;
  double *dense;     // nx*ny*nz*5 staging (caller layout)
  double *partial;   // integrals: 10 x nz
  double *extA, *extB;
  unsigned char *bandmask, *rext, *nostate, *touched;
  int *extmap, *srcmap, *counts, *blist, *cutlist, *flist[2];
  Region band{nullptr, 0};  // the band list of the last interaction step
  Region fluid[2] = {{nullptr, 0}, {nullptr, 0}};  // each fluid's brick list
  const Region whole{nullptr, 0};
  Ext3 *ext;
  Mix3 *mix;
  int ext_cap = 0, mix_cap = 0, nbricks = 0;
  int ntouched = 0;          // touched flags per fluid (the larger brick count)
  int fv_small[2] = {0, 0};  // brick shape of each fluid's current RK step
  int sms = 152;
  int max_substeps = 4096;
  Scal3 *sc = nullptr;
  Scal3 hs;
  double lf[2][3], smax[2];
  double t = 0.0;
  bool inited = false;
  std::string err;
  // profiling of the finite-volume stage
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  long long prof_launches = 0, prof_cells = 0, prof_open = 0, k_launch0 = 0;
  double prof_ms = 0.0;
  unsigned long long cells0 = 0, open0 = 0;
};

static int fail(sif3_ctx *c, int code, const std::string &m) {
  if (c) c->err = m;
  return code;
}

static int cuda_check(sif3_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SIF_OK;
  return fail(c, SIF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static double dt_of(const sif3_ctx *c, int k) {
  return c->smax[k] > 0.0 ? c->cfg.cfl / c->smax[k] : INFINITY;
}

static double bits_d(unsigned long long b) {
  double v;
  memcpy(&v, &b, sizeof v);
  return v;
}

// ---------------------------------------------------------------------
// memory: one pool, carved in 256-byte pieces

struct Carver {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    size_t b = (n * sizeof(T) + 255) & ~(size_t)255;
    T *p = base ? (T *)(base + off) : nullptr;
    off += b;
    return p;
  }
};

static void carve(sif3_ctx *c, Carver &cv) {
  size_t NP = (size_t)c->g.NP, n = (size_t)c->g.nx * c->g.ny * c->g.nz;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < S3_NC; m++) {
      c->q[k][m] = cv.take<double>(NP);
      c->w[k][m] = cv.take<double>(NP);
      c->q0[k][m] = cv.take<double>(NP);
    }
  for (int m = 0; m < S3_NC; m++) {
    c->prev[m] = cv.take<double>(NP);
    c->fut[m] = cv.take<double>(NP);
    c->qi[m] = cv.take<double>(NP);
  }
  for (int m = 0; m < 4; m++) {
    c->xc[m] = cv.take<double>(NP);
    c->xn[m] = cv.take<double>(NP);
    c->xp[m] = cv.take<double>(NP);
  }
  for (int d = 0; d < 3; d++) c->ul[d] = cv.take<double>(NP);
  double **one[] = {&c->phi, &c->phi0, &c->lphi, &c->p0, &c->old, &c->alpha, &c->ax,
                    &c->ay,  &c->az,   &c->sx,   &c->sy, &c->sz,  &c->corner};
  for (double **p : one) *p = cv.take<double>(NP);
  c->dense = cv.take<double>(n * S3_NC);
  c->partial = cv.take<double>((size_t)2 * S3_NC * c->g.nz);
  c->extA = cv.take<double>((size_t)3 * S3_NC * c->ext_cap);
  c->extB = cv.take<double>((size_t)3 * S3_NC * c->ext_cap);
  c->bandmask = cv.take<unsigned char>(NP);
  c->rext = cv.take<unsigned char>(NP);
  c->nostate = cv.take<unsigned char>(2 * NP);
  c->touched = cv.take<unsigned char>((size_t)2 * c->ntouched);
  c->extmap = cv.take<int>(3 * NP);
  c->srcmap = cv.take<int>(NP);
  c->counts = cv.take<int>(8);
  c->blist = cv.take<int>((size_t)c->nbricks);
  c->flist[0] = cv.take<int>((size_t)c->nbricks);
  c->flist[1] = cv.take<int>((size_t)c->nbricks);
  c->cutlist = cv.take<int>((size_t)c->ext_cap);
  c->ext = cv.take<Ext3>((size_t)3 * c->ext_cap);
  c->mix = cv.take<Mix3>((size_t)c->mix_cap);
  c->sc = cv.take<Scal3>(1);
}

static bool bc_ok(int b) { return b == SIF_BC_REFLECT || b == SIF_BC_ZEROGRAD || b == SIF_BC_PERIODIC; }

int sif3_create(const sif3_config *cfg, sif3_ctx **out) {
  if (!out) return SIF_EINVAL;
  *out = nullptr;
  if (!cfg) return SIF_EINVAL;
  const sif3_config &f = *cfg;
  if (f.nx < 3 || f.ny < 3 || f.nz < 3) return SIF_EINVAL;
  double np = (double)(f.nx + 6) * (f.ny + 6) * (f.nz + 6);
  if (np >= 2147483647.0) return SIF_EINVAL;
  if (!(f.dx > 0) || !(f.dy > 0) || !(f.dz > 0) || !(f.cfl > 0) || !(f.weno_eps >= 1e-20))
    return SIF_EINVAL;
  if (f.ext_iters < 0 || f.reinit_iters < 0 || !(f.band > 0) || !(f.mix_alpha > 0))
    return SIF_EINVAL;
  if (!(f.sigma >= 0.0) || !std::isfinite(f.sigma)) return SIF_EINVAL;
  for (int k = 0; k < 2; k++)
    if (!(f.mu[k] >= 0.0) || !std::isfinite(f.mu[k])) return SIF_EINVAL;
  for (int s = 0; s < 6; s++)
    if (!bc_ok(f.bc[s])) return SIF_EINVAL;
  for (int d = 0; d < 3; d++)
    if ((f.bc[2 * d] == SIF_BC_PERIODIC) != (f.bc[2 * d + 1] == SIF_BC_PERIODIC))
      return SIF_EINVAL;
  for (int k = 0; k < 2; k++) {
    if (!(f.gamma[k] > 1.0)) return SIF_EINVAL;
    if (f.tait[k] != 0 && f.tait[k] != 1) return SIF_EINVAL;
    if (f.tait[k] && (!(f.tait_B[k] > 0) || !(f.tait_rho0[k] > 0) || !std::isfinite(f.tait_p0[k])))
      return SIF_EINVAL;
  }
  sif3_ctx *c = new sif3_ctx();
  c->cfg = f;
  Grid3 &g = c->g;
  g.nx = f.nx, g.ny = f.ny, g.nz = f.nz;
  g.PX = f.nx + 2 * S3_GH, g.PY = f.ny + 2 * S3_GH, g.PZ = f.nz + 2 * S3_GH;
  g.NP = g.PX * g.PY * g.PZ;
  for (int s = 0; s < 6; s++) g.bc[s] = f.bc[s];
  g.dx = f.dx, g.dy = f.dy, g.dz = f.dz;
  g.h = fmin(fmin(f.dx, f.dy), f.dz);
  g.bw = f.band * g.h;
  for (int k = 0; k < 2; k++) {
    g.gamma[k] = f.gamma[k];
    g.tait[k] = f.tait[k];
    g.tB[k] = f.tait_B[k], g.tr0[k] = f.tait_rho0[k], g.tp0[k] = f.tait_p0[k];
    g.pinf[k] = f.tait[k] ? f.tait_B[k] - f.tait_p0[k] : f.pinf[k];
  }
  g.eps = f.weno_eps;
  g.mix_alpha = f.mix_alpha;
  g.sigma = f.sigma;
  g.mu[0] = f.mu[0];
  g.mu[1] = f.mu[1];
  g.newton_iters = 50;
  int n = f.nx * f.ny * f.nz;
  c->ext_cap = std::min(n, std::max(1 << 18, n / 4));
  c->mix_cap = std::min(n, std::max(1 << 16, n / 16));
  c->nbricks = ((f.nx + S3_BX - 1) / S3_BX) * ((f.ny + S3_BY - 1) / S3_BY) *
               ((f.nz + S3_BZ - 1) / S3_BZ);
  int rc = cuda_check(c, cudaSetDevice(f.device), "cudaSetDevice");
  if (rc) {
    delete c;
    return rc;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, f.device);
  c->ntouched = std::max(c->nbricks, k3_fv_bricks(g, 1));
  if (f.cuda_stream) {
    c->st = (cudaStream_t)f.cuda_stream;
  } else {
    if (cudaStreamCreate(&c->st) != cudaSuccess) {
      delete c;
      return SIF_ECUDA;
    }
    c->own_stream = true;
  }
  Carver dry{nullptr};
  carve(c, dry);
  c->pool_bytes = dry.off;
  if (cudaMalloc(&c->pool, c->pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
    return SIF_ECUDA;
  }
  Carver real{c->pool};
  carve(c, real);
  cudaMemsetAsync(c->pool, 0, c->pool_bytes, c->st);
  // the extension and mixing maps hold -1 between plans
  cudaMemsetAsync(c->extmap, 0xff, sizeof(int) * 3 * (size_t)c->g.NP, c->st);
  cudaMemsetAsync(c->srcmap, 0xff, sizeof(int) * (size_t)c->g.NP, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) {
    cudaFree(c->pool);
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
    return SIF_ECUDA;
  }
  *out = c;
  return SIF_OK;
}

int sif3_destroy(sif3_ctx *c) {
  if (!c) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  if (c->st) cudaStreamSynchronize(c->st);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  cudaFree(c->pool);
  if (c->own_stream) cudaStreamDestroy(c->st);
  delete c;
  return SIF_OK;
}

const char *sif3_last_error(const sif3_ctx *c) { return c ? c->err.c_str() : "null context"; }

// ---------------------------------------------------------------------
// pieces of the step

static void ghost1(sif3_ctx *c, double *p) {
  Planes3 s{};
  s.p[0] = p;
  s.n = 1;
  k3_launch_ghost(c->g, s, c->st);
}

static void ghost_w(sif3_ctx *c, int k) {
  Planes3 s{};
  for (int m = 0; m < S3_NC; m++) {
    s.p[m] = c->w[k][m];
    s.vel[m] = (m >= 1 && m <= 3) ? m : 0;
  }
  s.n = S3_NC;
  k3_launch_ghost(c->g, s, c->st);
}

// geometry of phi over the band list (the level set changed only there
// since the list was built), or over the whole grid
static void geometry(sif3_ctx *c, double *phi, bool all = false) {
  ghost1(c, phi);
  k3_launch_geometry(c->g, all ? c->whole : c->band, phi, c->corner, c->alpha, c->ax, c->ay,
                     c->az, c->sx, c->sy, c->sz, c->st);
}

// the band list from the current level set, its size read back
static int rebuild_band(sif3_ctx *c) {
  k3_launch_band_bricks(c->g, c->nbricks, c->phi, c->alpha, c->blist, c->flist[0],
                        c->flist[1], c->sc, c->st);
  int n[3] = {0, 0, 0};
  cudaMemcpyAsync(n, &c->sc->nband, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->st);
  int rc = cuda_check(c, cudaStreamSynchronize(c->st), "band list");
  c->band = Region{c->blist, n[0]};
  c->fluid[0] = Region{c->flist[0], n[1]};
  c->fluid[1] = Region{c->flist[1], n[2]};
  return rc;
}

static void copy_planes(sif3_ctx *c, double *const dst[], double *const src[], int n) {
  for (int m = 0; m < n; m++)
    cudaMemcpyAsync(dst[m], src[m], sizeof(double) * c->g.NP, cudaMemcpyDeviceToDevice, c->st);
}

// small cells lie near the interface: mixing works over the band list
static void mix(sif3_ctx *c, int k, double *const q[S3_NC]) {
  k3_launch_mix(c->g, c->band, k, q, c->alpha, c->phi, c->srcmap, c->mix, c->counts + 3,
                c->mix_cap, &c->sc->err, c->st);
}

// reads the device maxima and error bits after an interaction step
static int read_scalars(sif3_ctx *c) {
  cudaMemcpyAsync(&c->hs, c->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, c->st);
  int rc = cuda_check(c, cudaStreamSynchronize(c->st), "interaction step");
  if (rc) return rc;
  for (int k = 0; k < 2; k++) {
    for (int d = 0; d < 3; d++) c->lf[k][d] = bits_d(c->hs.lf[k][d]);
    c->smax[k] = bits_d(c->hs.smax[k]);
  }
  c->band = Region{c->blist, c->hs.nband};
  c->fluid[0] = Region{c->flist[0], c->hs.nfluid[0]};
  c->fluid[1] = Region{c->flist[1], c->hs.nfluid[1]};
  if (c->hs.err & S3_ERR_CAP)
    return fail(c, SIF_EINVAL, "a band list outgrew its capacity (interface too large for "
                               "the grid's band lists)");
  if (c->hs.err & S3_ERR_NONPHYS)
    return fail(c, SIF_ENONPHYS, "non-physical state (rho <= 0 or p + p_inf <= 0) in a full cell");
  if (c->hs.err & S3_ERR_NOCONV)
    return fail(c, SIF_ENOCONV, "interface Riemann Newton iteration did not converge");
  return SIF_OK;
}

// the interaction step for stage states qs and the level set (Sec. 2.1,
// 2.3): geometry, stencil states with extension, wave maxima, the
// interface Riemann problems, the level-set velocity; then the band list
// for the next stage.  band_only = f marks an evaluation inside the
// accelerated cycle whose fluid-1 states (f) are read only near the
// interface (its stencil states elsewhere, its time step and its
// Lax-Friedrichs speeds are not used before they are evaluated again over
// its brick list); -1 evaluates each fluid over its brick list
static int eval(sif3_ctx *c, double *const qs[2][S3_NC], double *phi, int band_only = -1) {
  const Grid3 &g = c->g;
  geometry(c, phi);
  cudaMemsetAsync(c->sc, 0, offsetof(Scal3, err), c->st);  // maxima restart, errors stick
  // each fluid's cells lie in its brick list (built with the band list
  // at the previous interaction step)
  for (int k = 0; k < 2; k++)
    k3_launch_prim(g, k == band_only ? c->band : c->fluid[k], k, qs[k], c->w[k], c->alpha,
                   c->nostate, c->sc, c->st);
  k3_ext_plan(g, c->band, 0, phi, c->alpha, c->nostate, c->sx, c->sy, c->sz, c->extmap, c->ext,
              c->counts, c->ext_cap, &c->sc->err, c->st);
  double *wp[2 * S3_NC];
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < S3_NC; m++) wp[k * S3_NC + m] = c->w[k][m];
  k3_launch_ext_sweeps(g, 0, c->cfg.ext_iters, c->ext, c->counts, c->ext_cap, wp, S3_NC,
                       c->extA, c->extB, c->extmap, c->st);
  for (int k = 0; k < 2; k++)
    if (k != band_only)
      k3_launch_wave_maxima(g, c->fluid[k], k, c->w[k], c->alpha, c->nostate, phi, c->sc,
                            c->st);
  if (g.mu[0] > 0.0 && g.mu[1] > 0.0) {
    // the traction's central differences reach the ghost layers
    Planes3 v{};
    for (int k = 0; k < 2; k++)
      for (int b = 0; b < 3; b++) {
        v.p[3 * k + b] = c->w[k][1 + b];
        v.vel[3 * k + b] = 1 + b;
      }
    v.n = 6;
    k3_launch_ghost(g, v, c->st);
  }
  k3_launch_interface(g, c->band, c->w, phi, c->sx, c->sy, c->sz, c->xn, c->xp, c->ul,
                      c->cutlist, c->counts + 4, c->ext_cap, c->sc, c->st);
  k3_ext_plan(g, c->band, 2, phi, c->alpha, c->nostate, c->sx, c->sy, c->sz, c->extmap, c->ext,
              c->counts, c->ext_cap, &c->sc->err, c->st);
  k3_launch_ext_sweeps(g, 2, c->cfg.ext_iters, c->ext, c->counts, c->ext_cap, c->ul, 3,
                       c->extA, c->extB, c->extmap, c->st);
  k3_launch_band_bricks(g, c->nbricks, phi, c->alpha, c->blist, c->flist[0], c->flist[1], c->sc,
                        c->st);
  return read_scalars(c);
}

static void fv(sif3_ctx *c, int k, int stage, double dt, double *const dst[S3_NC],
               double *const cur[S3_NC], double *const base[S3_NC]) {
  ghost_w(c, k);
  Fv3Args a{};
  // a fluid on fewer bricks than one wave of the stage's CTAs (three per
  // SM) runs on 4 x 4 x 4 bricks: its launch lasts about one CTA's
  // lifetime, which the smaller bricks shorten; the shape is kept from
  // stage 1 to stage 2 (the touched flags are per brick)
  if (stage == 1) c->fv_small[k] = c->fluid[k].count < 3 * c->sms ? 1 : 0;
  a.touched = c->touched + (size_t)k * c->ntouched;
  a.k = k;
  a.stage = stage;
  a.dt = dt;
  for (int d = 0; d < 3; d++) a.lf[d] = c->lf[k][d];
  for (int m = 0; m < S3_NC; m++) {
    a.w[m] = c->w[k][m];
    a.dst[m] = dst[m];
    a.cur[m] = cur[m];
    a.base[m] = base ? base[m] : cur[m];
  }
  a.ax = c->ax, a.ay = c->ay, a.az = c->az;
  for (int m = 0; m < 4; m++) a.x[m] = k ? c->xp[m] : c->xn[m];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    if (c->ev_used + 2 > c->ev.size()) {
      for (int q = 0; q < 64; q++) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev.push_back(e);
      }
    }
    e0 = c->ev[c->ev_used++];
    e1 = c->ev[c->ev_used++];
    cudaEventRecord(e0, c->st);
  }
  k3_launch_fv(c->g, a, c->sc, c->st, c->fv_small[k]);
  if (c->g.mu[k] > 0.0) k3_launch_viscous(c->g, a, c->st);
  if (c->prof) {
    cudaEventRecord(e1, c->st);
    c->prof_launches++;
  }
}

// level-set RK stage over the band of phi0
static void ls_stage(sif3_ctx *c, int stage, double dt) {
  ghost1(c, c->phi);
  k3_launch_ls_rhs(c->g, c->band, c->phi, c->ul, c->bandmask, c->lphi, c->st);
  k3_launch_rk(c->g, c->band, stage, c->phi, c->phi0, c->lphi, dt, c->bandmask, c->st);
}

static void reinit(sif3_ctx *c) {
  ghost1(c, c->phi);
  cudaMemcpyAsync(c->p0, c->phi, sizeof(double) * c->g.NP, cudaMemcpyDeviceToDevice, c->st);
  for (int it = 0; it < c->cfg.reinit_iters; it++) {
    ghost1(c, c->phi);
    cudaMemcpyAsync(c->old, c->phi, sizeof(double) * c->g.NP, cudaMemcpyDeviceToDevice, c->st);
    k3_launch_reinit(c->g, c->band, c->phi, c->old, c->p0, c->rext, c->st);
  }
}

static void start_level_set_step(sif3_ctx *c) {
  cudaMemcpyAsync(c->phi0, c->phi, sizeof(double) * c->g.NP, cudaMemcpyDeviceToDevice, c->st);
  k3_launch_band(c->g, c->phi0, c->bandmask, c->rext, c->st);
}

// one RK2 step of both fluids and the level set with a common dt, the
// first interaction step evaluated already
static int single_step_after_eval(sif3_ctx *c, double dt) {
  for (int k = 0; k < 2; k++) copy_planes(c, c->q0[k], c->q[k], S3_NC);
  start_level_set_step(c);
  for (int s = 1; s <= 2; s++) {
    if (s > 1) {
      int rc = eval(c, c->q, c->phi);
      if (rc) return rc;
    }
    for (int k = 0; k < 2; k++) fv(c, k, s, dt, c->q[k], c->q[k], c->q0[k]);
    ls_stage(c, s, dt);
    if (s == 2) reinit(c);
    geometry(c, c->phi);
    mix(c, 0, c->q[0]);
    mix(c, 1, c->q[1]);
  }
  c->t += dt;
  return SIF_OK;
}

// one accelerated cycle (Sec. 3.1, steps 1-5) with TVD-RK2
static int cycle(sif3_ctx *c, double t_end, sif_cycle_info *info) {
  int rc = eval(c, c->q, c->phi);
  if (rc) return rc;
  double dtk[2] = {dt_of(c, 0), dt_of(c, 1)};
  for (int k = 0; k < 2; k++)
    if (t_end > 0.0 && c->t + dtk[k] > t_end) dtk[k] = t_end - c->t;
  int f1 = dtk[1] > dtk[0] ? 1 : 0, f2 = 1 - f1;
  double dt1 = dtk[f1], dt2 = dtk[f2];
  double nraw = dt1 / dt2;
  if (info) {
    info->n_raw = nraw;
    info->role_fluid1 = f1;
    info->dt2 = dt2;
  }
  if (c->cfg.force_ratio_one) {
    dt1 = dt2;
  } else {
    if (std::isfinite(dt1)) {
      double fl = floor(nraw);
      if (nraw - fl < c->cfg.ratio_threshold) dt1 = fl * dt2;
    }
    if (!std::isfinite(dt1) || dt1 <= dt2) {
      rc = single_step_after_eval(c, dt2);
      if (info) {
        info->dt1 = dt2;
        info->n_used = 1.0;
        info->substeps = 1;
        info->t = c->t;
      }
      return rc;
    }
  }
  if (info) {
    info->dt1 = dt1;
    info->n_used = dt1 / dt2;
  }
  for (int m = 0; m < 4; m++) cudaMemsetAsync(c->xc[m], 0, sizeof(double) * c->g.NP, c->st);
  double *const *x1 = f1 == 0 ? c->xn : c->xp;
  // step 2: fluid 1's first stage with dt1 into fut; prev keeps t^n
  copy_planes(c, c->prev, c->q[f1], S3_NC);
  copy_planes(c, c->fut, c->prev, S3_NC);
  fv(c, f1, 1, dt1, c->fut, c->fut, nullptr);
  double t2 = 0.0;
  int sub = 0;
  double *qs[2][S3_NC];
  for (;;) {
    sub++;
    if (sub > c->max_substeps)
      return fail(c, SIF_ETIMEOUT, "sub-cycle loop reached its limit of " +
                                       std::to_string(c->max_substeps) + " sub-steps");
    if (sub > 1) {
      k3_launch_interp(c->g, c->band, c->qi, c->prev, c->fut, t2 / dt1, c->st);
      geometry(c, c->phi);
      mix(c, f1, c->qi);
      for (int m = 0; m < S3_NC; m++) {
        qs[f1][m] = c->qi[m];
        qs[f2][m] = c->q[f2][m];
      }
      rc = eval(c, qs, c->phi, f1);
      if (rc) return rc;
      dt2 = dt_of(c, f2);
    }
    bool last = (dt1 - t2) <= dt2 * (1.0 + 1e-12);
    if (last) dt2 = dt1 - t2;
    k3_launch_record(c->g, c->band, sub == 1, x1, c->xc, dt1, dt2, c->st);
    // step 3: fluid 2 and the level set, first stage with dt2
    copy_planes(c, c->q0[f2], c->q[f2], S3_NC);
    start_level_set_step(c);
    fv(c, f2, 1, dt2, c->q[f2], c->q[f2], nullptr);
    ls_stage(c, 1, dt2);
    geometry(c, c->phi);
    mix(c, f2, c->q[f2]);
    if (last) {
      mix(c, f1, c->fut);
      for (int m = 0; m < S3_NC; m++) qs[f1][m] = c->fut[m];
    } else {
      k3_launch_interp(c->g, c->band, c->qi, c->prev, c->fut, (t2 + dt2) / dt1, c->st);
      mix(c, f1, c->qi);
      for (int m = 0; m < S3_NC; m++) qs[f1][m] = c->qi[m];
    }
    for (int m = 0; m < S3_NC; m++) qs[f2][m] = c->q[f2][m];
    rc = eval(c, qs, c->phi, last ? -1 : f1);
    if (rc) return rc;
    k3_launch_record(c->g, c->band, last, x1, c->xc, dt1, dt2, c->st);
    // step 4 (and 5 on the last sub-step): second stage
    fv(c, f2, 2, dt2, c->q[f2], c->q[f2], c->q0[f2]);
    ls_stage(c, 2, dt2);
    if (last) fv(c, f1, 2, dt1, c->q[f1], c->fut, c->prev);
    reinit(c);
    if (last) {
      if (c->cfg.flux_correction)
        k3_launch_correction(c->g, c->q[f1], c->xc, c->g.dx * c->g.dy * c->g.dz, c->st);
      geometry(c, c->phi);
      mix(c, f1, c->q[f1]);
      mix(c, f2, c->q[f2]);
      break;
    }
    t2 += dt2;
    geometry(c, c->phi);
    mix(c, f2, c->q[f2]);
  }
  c->t += dt1;
  if (info) {
    info->substeps = sub;
    info->t = c->t;
  }
  return SIF_OK;
}

static void counters_start(sif3_ctx *c) {
  cudaMemcpyAsync(&c->hs, c->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  c->cells0 = c->hs.cells;
  c->open0 = c->hs.open;
}

static int finish(sif3_ctx *c, int rc, sif_cycle_info *info) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (!rc && e != cudaSuccess) rc = cuda_check(c, e, "step");
  cudaMemcpy(&c->hs, c->sc, sizeof(Scal3), cudaMemcpyDeviceToHost);
  if (info) {
    info->cell_updates = (long long)(c->hs.cells - c->cells0);
    info->open_updates = (long long)(c->hs.open - c->open0);
  }
  if (!rc && (c->hs.err & S3_ERR_CAP)) rc = fail(c, SIF_EINVAL, "a band list outgrew its capacity");
  if (!rc && (c->hs.err & S3_ERR_NONPHYS)) rc = fail(c, SIF_ENONPHYS, "non-physical state");
  return rc;
}

int sif3_step_single_dt(sif3_ctx *c, int nsteps, double t_end, sif_cycle_info *info) {
  if (!c) return SIF_EINVAL;
  if (!c->inited) return fail(c, SIF_ESTATE, "step before sif3_init_fluids");
  if (nsteps < 0) return fail(c, SIF_EINVAL, "nsteps < 0");
  cudaSetDevice(c->cfg.device);
  counters_start(c);
  int rc = SIF_OK;
  for (int n = 0; n < nsteps && !rc; n++) {
    if (t_end > 0.0 && c->t >= t_end) break;
    rc = eval(c, c->q, c->phi);
    if (rc) break;
    double dt = std::min(dt_of(c, 0), dt_of(c, 1));
    if (t_end > 0.0 && c->t + dt > t_end) dt = t_end - c->t;
    if (!std::isfinite(dt)) {
      rc = fail(c, SIF_EINVAL, "no fluid limits the time step");
      break;
    }
    rc = single_step_after_eval(c, dt);
    if (info) {
      info->t = c->t;
      info->dt1 = info->dt2 = dt;
      info->n_raw = info->n_used = 1.0;
      info->role_fluid1 = -1;
      info->substeps = 1;
    }
  }
  return finish(c, rc, info);
}

int sif3_step_multi_dt(sif3_ctx *c, int ncycles, double t_end, sif_cycle_info *info) {
  if (!c) return SIF_EINVAL;
  if (!c->inited) return fail(c, SIF_ESTATE, "step before sif3_init_fluids");
  if (ncycles < 0) return fail(c, SIF_EINVAL, "ncycles < 0");
  cudaSetDevice(c->cfg.device);
  counters_start(c);
  int rc = SIF_OK;
  for (int n = 0; n < ncycles && !rc; n++) {
    if (t_end > 0.0 && c->t >= t_end) break;
    rc = cycle(c, t_end, info);
  }
  return finish(c, rc, info);
}

// ---------------------------------------------------------------------
// data in and out: the caller's dense (nz, ny, nx) planes through the
// staging buffer (host memory) or directly (device memory)

static size_t ncell(const sif3_ctx *c) { return (size_t)c->g.nx * c->g.ny * c->g.nz; }

static int planes_in(sif3_ctx *c, const double *src, int nplanes, double *const dst[],
                     int mem_kind) {
  size_t n = ncell(c);
  const double *d = src;
  if (mem_kind == SIF_HOST) {
    int rc = cuda_check(c, cudaMemcpyAsync(c->dense, src, sizeof(double) * n * nplanes,
                                           cudaMemcpyHostToDevice, c->st), "copy in");
    if (rc) return rc;
    d = c->dense;
  }
  for (int m = 0; m < nplanes; m++) k3_launch_pack(c->g, dst[m], (double *)d + m * n, 1, c->st);
  return SIF_OK;
}

static int planes_out(sif3_ctx *c, double *dst, int nplanes, double *const src[],
                      int mem_kind) {
  size_t n = ncell(c);
  double *d = mem_kind == SIF_HOST ? c->dense : dst;
  for (int m = 0; m < nplanes; m++) k3_launch_pack(c->g, src[m], d + m * n, 0, c->st);
  if (mem_kind == SIF_HOST)
    cudaMemcpyAsync(dst, c->dense, sizeof(double) * n * nplanes, cudaMemcpyDeviceToHost, c->st);
  return cuda_check(c, cudaStreamSynchronize(c->st), "copy out");
}

static bool kind_ok(int k) { return k == SIF_HOST || k == SIF_DEVICE; }

int sif3_init_fluids(sif3_ctx *c, const double *phi, const double *pN, const double *pP,
                     int mem_kind) {
  if (!c) return SIF_EINVAL;
  if (!phi || !pN || !pP || !kind_ok(mem_kind)) return fail(c, SIF_EINVAL, "bad arguments");
  cudaSetDevice(c->cfg.device);
  double *one[1] = {c->phi};
  int rc = planes_in(c, phi, 1, one, mem_kind);
  if (rc) return rc;
  geometry(c, c->phi, true);
  rc = rebuild_band(c);
  if (rc) return rc;
  size_t n = ncell(c);
  for (int k = 0; k < 2; k++) {
    const double *src = k ? pP : pN;
    const double *d = src;
    if (mem_kind == SIF_HOST) {
      cudaMemcpyAsync(c->dense, src, sizeof(double) * n * S3_NC, cudaMemcpyHostToDevice, c->st);
      d = c->dense;
    }
    k3_launch_init_state(c->g, c->alpha, d, c->q[k], c->w[k], k, c->st);
  }
  cudaMemsetAsync(&c->sc->err, 0, sizeof(int), c->st);
  mix(c, 0, c->q[0]);
  mix(c, 1, c->q[1]);
  c->t = 0.0;
  rc = cuda_check(c, cudaStreamSynchronize(c->st), "init");
  if (rc) return rc;
  c->inited = true;
  return SIF_OK;
}

int sif3_get_state(sif3_ctx *c, double *qN, double *qP, double *phi, int mem_kind) {
  if (!c) return SIF_EINVAL;
  if (!kind_ok(mem_kind)) return fail(c, SIF_EINVAL, "bad mem_kind");
  cudaSetDevice(c->cfg.device);
  int rc = SIF_OK;
  if (qN) rc = planes_out(c, qN, S3_NC, c->q[0], mem_kind);
  if (!rc && qP) rc = planes_out(c, qP, S3_NC, c->q[1], mem_kind);
  double *one[1] = {c->phi};
  if (!rc && phi) rc = planes_out(c, phi, 1, one, mem_kind);
  return rc;
}

int sif3_set_state(sif3_ctx *c, const double *qN, const double *qP, const double *phi,
                   int mem_kind) {
  if (!c) return SIF_EINVAL;
  if (!kind_ok(mem_kind)) return fail(c, SIF_EINVAL, "bad mem_kind");
  cudaSetDevice(c->cfg.device);
  int rc = SIF_OK;
  if (qN) rc = planes_in(c, qN, S3_NC, c->q[0], mem_kind);
  if (!rc && qP) rc = planes_in(c, qP, S3_NC, c->q[1], mem_kind);
  double *one[1] = {c->phi};
  if (!rc && phi) rc = planes_in(c, phi, 1, one, mem_kind);
  if (rc) return rc;
  // a state set from outside starts without the error bits of the last step
  cudaMemsetAsync(&c->sc->err, 0, sizeof(int), c->st);
  geometry(c, c->phi, true);
  rc = rebuild_band(c);
  if (rc) return rc;
  c->inited = true;
  return cuda_check(c, cudaStreamSynchronize(c->st), "set state");
}

int sif3_integrals(sif3_ctx *c, double *out) {
  if (!c || !out) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  k3_launch_integrals(c->g, c->q, c->partial, c->st);
  std::vector<double> h((size_t)2 * S3_NC * c->g.nz);
  cudaMemcpyAsync(h.data(), c->partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st);
  int rc = cuda_check(c, cudaStreamSynchronize(c->st), "integrals");
  if (rc) return rc;
  double dv = c->g.dx * c->g.dy * c->g.dz;
  for (int q = 0; q < 2 * S3_NC; q++) {
    double s = 0.0;
    for (int z = 0; z < c->g.nz; z++) s += h[(size_t)q * c->g.nz + z];
    out[q] = s * dv;
  }
  return SIF_OK;
}

int sif3_geometry(sif3_ctx *c, double *alpha, double *ax, double *ay, double *az, double *sx,
                  double *sy, double *sz, int mem_kind) {
  if (!c) return SIF_EINVAL;
  if (!kind_ok(mem_kind)) return fail(c, SIF_EINVAL, "bad mem_kind");
  cudaSetDevice(c->cfg.device);
  geometry(c, c->phi, true);
  double *outs[7] = {alpha, ax, ay, az, sx, sy, sz};
  double *srcs[7] = {c->alpha, c->ax, c->ay, c->az, c->sx, c->sy, c->sz};
  for (int q = 0; q < 7; q++) {
    if (!outs[q]) continue;
    int rc = planes_out(c, outs[q], 1, &srcs[q], mem_kind);
    if (rc) return rc;
  }
  return SIF_OK;
}

int sif3_set_limits(sif3_ctx *c, int max_substeps, int newton_iters) {
  if (!c) return SIF_EINVAL;
  if (max_substeps > 1000000 || newton_iters > 10000)
    return fail(c, SIF_EINVAL, "limits above 1000000 sub-steps or 10000 iterations");
  if (max_substeps > 0) c->max_substeps = max_substeps;
  if (newton_iters > 0) c->g.newton_iters = newton_iters;
  return SIF_OK;
}

int sif3_get_time(const sif3_ctx *c, double *t) {
  if (!c || !t) return SIF_EINVAL;
  *t = c->t;
  return SIF_OK;
}

int sif3_profile_enable(sif3_ctx *c, int on) {
  if (!c) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  cudaStreamSynchronize(c->st);
  c->prof = on != 0;
  c->ev_used = 0;
  c->prof_launches = 0;
  c->prof_ms = 0.0;
  c->k_launch0 = (long long)(k3_launches() + k3_fv_launches());
  cudaMemcpy(&c->hs, c->sc, sizeof(Scal3), cudaMemcpyDeviceToHost);
  c->cells0 = c->hs.cells;
  c->open0 = c->hs.open;
  c->prof_cells = (long long)c->hs.cells;
  c->prof_open = (long long)c->hs.open;
  return SIF_OK;
}

int sif3_profile_read(sif3_ctx *c, sif_profile *out) {
  if (!c || !out) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  int rc = cuda_check(c, cudaStreamSynchronize(c->st), "profile");
  if (rc) return rc;
  double ms = 0.0;
  for (size_t e = 0; e + 1 < c->ev_used; e += 2) {
    float m = 0.f;
    cudaEventElapsedTime(&m, c->ev[e], c->ev[e + 1]);
    ms += m;
  }
  cudaMemcpy(&c->hs, c->sc, sizeof(Scal3), cudaMemcpyDeviceToHost);
  out->kernel_launches = (long long)(k3_launches() + k3_fv_launches()) - c->k_launch0;
  out->fv_launches = c->prof_launches;
  out->fv_ms = ms;
  out->fv_cell_updates = (long long)c->hs.cells - c->prof_cells;
  out->fv_open_updates = (long long)c->hs.open - c->prof_open;
  c->ev_used = 0;
  c->prof_launches = 0;
  c->k_launch0 = (long long)(k3_launches() + k3_fv_launches());
  c->prof_cells = (long long)c->hs.cells;
  c->prof_open = (long long)c->hs.open;
  return SIF_OK;
}
