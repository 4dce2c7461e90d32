// api.cu -- the C-ABI of libsif (include/sif.h): context and device memory,
// and the host-side sequencing of the kernels for the original
// single-time-step method and for one cycle of the accelerated method
// (Sec. 3.1, steps 1-5).  Every arithmetic step runs in the kernels; the
// host only orders launches and, once per fluid-2 sub-step, reads back the
// scheduler's branch decision.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <stddef.h>
#include <new>
#include <vector>

#include "sif_internal.cuh"

struct sif_ctx {
  sif_config cfg;
  Grid g;
  cudaStream_t st;
  size_t NP;
  // xn: exchange flux as applied to fluid N; xm: as applied to fluid P,
  // negated (equal to xn without surface tension and viscosity)
  double *q[2][4], *w[2][4], *phi, *alpha, *ax, *ay, *sx, *sy, *xn[3], *xm[3], *ul[2];
  double *q0[2][4], *prev[4], *fut[4], *qi[4], *xc[3], *phi0, *phiR;
  double *phia, *phib, *phie;  // RK3 cycle: kept level sets (see graph_cycle_body3)
  double *tmp;       // band-indexed scratch, 8 planes
  int *bandmap;      // cell -> position in the interaction band, -1 outside
  ExtPlan *ext_plan; // 3 x ncell
  MixPlan *mix_plan; // 2 x ncell
  int band_work;     // recent interaction-band size, sizes band grids
  double *partial;   // integrals: 8*ny partial sums + pointer table
  double *integ;     // 8 totals
  int *band_ev, *band_ls, *rext_ls, *cut, *tiles[2];
  int *etiles;       // band tiles of the blocked extension
  unsigned char *nostate[2];  // per fluid: cut cells holding no physical state
  Scalars *sc;       // device
  Scalars *hsc;      // pinned host mirror
  double *hbuf;      // pinned 8 doubles
  void *pool;        // single device allocation
  size_t pool_bytes;
  int debug_sync;    // SIF_DEBUG_SYNC=1: synchronise and check after each phase
  // profiling: device counters (kernel launches, finite-volume launch time)
  int profiling;
  unsigned long long launches0, updates0, open0;
  // work stream: the caller's, or a private blocking stream (ordered with
  // the legacy default stream) when the caller passes none
  cudaStream_t own_stream;
  // device-driven cycle graphs (conditional nodes) and capture state
  cudaStream_t cap[4];
  int cap_depth, capturing, gerr;
  // graph branch of the level-set velocity's extension: captured after the
  // interface interaction beside what follows, joined after the next
  // finite-volume launch (the capture's dependency set is saved before
  // the branch and restored after it; the branch's tail is added back at
  // the join)
  cudaGraphNode_t br_base[8], br_tail[8];
  cudaGraphEdgeData br_base_ed[8], br_tail_ed[8];
  size_t br_nbase, br_ntail;
  int br_base_has_ed, br_tail_has_ed;
  int side_pending;
  int use_graphs;
  int no_graph_env;    // SIF_NO_GRAPH=1: cycles issued from the host on purpose
  int ext_blocked;     // extension sweeps in shared memory per band tile (else one
                       // launch per sweep or two: batch instances, or
                       // SIF_EXT_SWEEPS=1)
  int require_graphs;  // SIF_REQUIRE_GRAPHS=1: a failed capture is an error
  int graph_bucket;  // band grid size baked into the graphs
  int num_sms;
  cudaGraphExec_t g_cycle, g_single;
  cudaGraph_t g_cycle_tmpl;  // kept for embedding in batch graphs
  int graph_gen;             // bumped whenever the graphs are rebuilt
  int inited;
  int last_status;
  int max_substeps;  // fluid-2 sub-steps allowed in one accelerated cycle
  // adjoint: tape of recorded single-time-step steps (own allocation) and
  // the adjoint's scratch planes (allocated on first use)
  int tape_cap, tape_len, tape_alloc;
  double *tape_planes;  // tape_alloc x kTapePlanes planes
  double *tape_scal;    // tape_alloc x 16: dt, LF speeds of stage 1 and 2 (bit patterns)
  void *adj_pool;
  double *lamA[2][4], *lamB[2][4], *lamC[2][4], *lw[2][4], *prim[2][4], *G[40];
  double *SP[8];  // split fluxes of one (fluid, direction) for the face coefficients
  double *sv_q[2][4], *sv_w[2][4], *sv_phi;
  Scalars *sv_sc;
  char err[256];
};

// per recorded step: q (8), the stencil states the step starts from (8),
// phi^n, phi after stage 1, phi^{n+1}, the stencil states (ghosts filled)
// that stage 1 and stage 2 used (8 + 8), and one plane holding, as bytes,
// the cut cells without a physical state of both stages and fluids
static const int kTapePlanes = 36;
static const int kTapeW1 = 19, kTapeW2 = 27, kTapeFlags = 35;

// default limits of the two bounded loops of a step (sif_set_limits)
static const int kMaxSubsteps = 4096;  // fluid-2 sub-steps in one cycle
static const int kNewtonMax = 50;      // Newton iterations per interface Riemann problem

// launch counting happens on the device (SIF_TICK); the host-side notes
// the wrappers make are not used for measurement
void sif_note_launches(int) {}
static unsigned long long device_launches() {
  return sif_launches_geom() + sif_launches_band() + sif_launches_plan() + sif_launches_fv() +
         sif_launches_adj();
}

static void set_err(sif_ctx *c, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
}

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      set_err(c, "%s: %s", #call, cudaGetErrorString(e_));                    \
      return SIF_ECUDA;                                                       \
    }                                                                         \
  } while (0)

static int ensure_graphs(sif_ctx *c);
static void free_graphs(sif_ctx *c);

static int check_launch(sif_ctx *c, const char *where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(c, "%s: %s", where, cudaGetErrorString(e));
    return SIF_ECUDA;
  }
  return SIF_OK;
}

static int validate(const sif_config *f, char *why, size_t n) {
  if (f->dim != 1 && f->dim != 2) return snprintf(why, n, "dim must be 1 or 2"), SIF_EINVAL;
  if (f->nx < 3) return snprintf(why, n, "nx must be >= 3"), SIF_EINVAL;
  if (f->dim == 1 && f->ny != 1) return snprintf(why, n, "dim 1 requires ny == 1"), SIF_EINVAL;
  if (f->dim == 2 && f->ny < 3) return snprintf(why, n, "ny must be >= 3"), SIF_EINVAL;
  if ((long long)(f->nx + 2 * SIF_GH) * (f->ny + 2 * SIF_GH) > (1ll << 31) / 4)
    return snprintf(why, n, "grid too large for 32-bit cell indices"), SIF_EINVAL;
  if (!(f->dx > 0.0) || !(f->dy > 0.0)) return snprintf(why, n, "dx, dy must be > 0"), SIF_EINVAL;
  for (int k = 0; k < 2; k++) {
    if (!(f->gamma[k] > 1.0)) return snprintf(why, n, "gamma must be > 1"), SIF_EINVAL;
    if (f->tait[k] != 0 && f->tait[k] != 1) return snprintf(why, n, "tait must be 0 or 1"), SIF_EINVAL;
    if (f->tait[k]) {
      if (!(f->tait_B[k] > 0.0 && f->tait_B[k] < 1e300) || !(f->tait_rho0[k] > 0.0 && f->tait_rho0[k] < 1e300) ||
          !(f->tait_p0[k] > -1e300 && f->tait_p0[k] < 1e300))
        return snprintf(why, n, "Tait parameters: B > 0, rho0 > 0, p0 finite"), SIF_EINVAL;
      if (f->weno_char) return snprintf(why, n, "weno_char requires stiffened-gas fluids"), SIF_EINVAL;
    } else if (!(f->pinf[k] >= 0.0)) {
      return snprintf(why, n, "p_inf must be >= 0"), SIF_EINVAL;
    }
  }
  for (int s = 0; s < 4; s++)
    if (f->bc[s] < 0 || f->bc[s] > 2) return snprintf(why, n, "bad boundary kind"), SIF_EINVAL;
  if ((f->bc[0] == SIF_BC_PERIODIC) != (f->bc[1] == SIF_BC_PERIODIC) ||
      (f->dim == 2 && (f->bc[2] == SIF_BC_PERIODIC) != (f->bc[3] == SIF_BC_PERIODIC)))
    return snprintf(why, n, "periodic boundaries must be paired"), SIF_EINVAL;
  if (!(f->cfl > 0.0) || f->cfl > 1.0) return snprintf(why, n, "cfl must be in (0, 1]"), SIF_EINVAL;
  if (f->rk_order != 2 && f->rk_order != 3) return snprintf(why, n, "rk_order must be 2 or 3"), SIF_EINVAL;
  if (f->weno_char != 0 && f->weno_char != 1) return snprintf(why, n, "weno_char must be 0 or 1"), SIF_EINVAL;
  if (f->flux != 0 && f->flux != 1) return snprintf(why, n, "flux must be 0 or 1"), SIF_EINVAL;
  if (f->flux == 1 && f->weno_char)
    return snprintf(why, n, "the HLLC flux reconstructs primitive states (weno_char 0)"), SIF_EINVAL;
  if (!(f->sigma >= 0.0 && f->sigma < 1e300)) return snprintf(why, n, "sigma must be finite and >= 0"), SIF_EINVAL;
  for (int k = 0; k < 2; k++)
    if (!(f->mu[k] >= 0.0 && f->mu[k] < 1e300)) return snprintf(why, n, "mu must be finite and >= 0"), SIF_EINVAL;
  // the face values' reciprocal needs the product of two denominators,
  // each at least eps^4, to stay normal
  if (!(f->weno_eps >= 1e-20)) return snprintf(why, n, "weno_eps must be >= 1e-20"), SIF_EINVAL;
  if (!(f->mix_alpha >= 0.0 && f->mix_alpha <= 1.0)) return snprintf(why, n, "mix_alpha in [0,1]"), SIF_EINVAL;
  if (!(f->ratio_threshold >= 0.0 && f->ratio_threshold <= 1.0))
    return snprintf(why, n, "ratio_threshold in [0,1]"), SIF_EINVAL;
  if (f->ext_iters < 1 || f->ext_iters > 1000) return snprintf(why, n, "ext_iters in [1,1000]"), SIF_EINVAL;
  if (f->reinit_iters < 0 || f->reinit_iters > 1000) return snprintf(why, n, "reinit_iters in [0,1000]"), SIF_EINVAL;
  if (!(f->band >= 3.0)) return snprintf(why, n, "band must be >= 3 cells"), SIF_EINVAL;
  return SIF_OK;
}

extern "C" int sif_create(const sif_config *cfg, sif_ctx **out) {
  if (!out) return SIF_EINVAL;
  *out = nullptr;
  if (!cfg) return SIF_EINVAL;
  sif_ctx *c = new (std::nothrow) sif_ctx();
  if (!c) return SIF_ECUDA;
  c->cfg = *cfg;
  char why[200];
  int rc = validate(cfg, why, sizeof(why));
  if (rc) {
    // the context is freed; the reason is unavailable to the caller here
    delete c;
    return rc;
  }
  sif_config &f = c->cfg;
  if (f.dim == 1) f.bc[2] = f.bc[3] = SIF_BC_ZEROGRAD;
  if (cudaSetDevice(f.device) != cudaSuccess) {
    delete c;
    return SIF_ECUDA;
  }
  c->st = (cudaStream_t)f.cuda_stream;
  if (!c->st) {
    if (cudaStreamCreate(&c->own_stream) != cudaSuccess) {
      delete c;
      return SIF_ECUDA;
    }
    c->st = c->own_stream;
  }
  for (int i = 0; i < 4; i++) cudaStreamCreateWithFlags(&c->cap[i], cudaStreamNonBlocking);
  fv_prepare();
  ext_prepare();
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->num_sms = sms > 0 ? sms : 1;
  }
  {
    const char *ng = getenv("SIF_NO_GRAPH");
    c->no_graph_env = ng && ng[0] == '1';
    c->use_graphs = !c->no_graph_env;
    const char *rq = getenv("SIF_REQUIRE_GRAPHS");
    c->require_graphs = rq && rq[0] == '1';
  }
  Grid &g = c->g;
  g.dim = f.dim;
  g.nx = f.nx;
  g.ny = f.ny;
  g.PX = ((f.nx + 2 * SIF_GH) + 15) / 16 * 16;
  g.PY = f.ny + 2 * SIF_GH;
  g.dx = f.dx;
  g.dy = f.dy;
  g.h = f.dim == 2 ? (f.dx < f.dy ? f.dx : f.dy) : f.dx;
  for (int s = 0; s < 4; s++) g.bc[s] = f.bc[s];
  for (int k = 0; k < 2; k++) {
    g.gamma[k] = f.gamma[k];
    g.pinf[k] = f.pinf[k];
    g.tait[k] = f.tait[k];
    g.tB[k] = f.tait_B[k];
    g.trho0[k] = f.tait_rho0[k];
    g.tp0[k] = f.tait_p0[k];
    // a Tait fluid's sound speed is the stiffened gas's with p_inf = B - p0
    if (f.tait[k]) g.pinf[k] = f.pinf[k] = f.tait_B[k] - f.tait_p0[k];
  }
  g.cfl = f.cfl;
  g.weno_eps = f.weno_eps;
  g.mix_alpha = f.mix_alpha;
  g.band = f.band;
  g.ext_iters = f.ext_iters;
  g.reinit_iters = f.reinit_iters;
  g.weno_char = f.weno_char;
  g.flux = f.flux;
  g.sigma = f.sigma;
  g.mu[0] = f.mu[0];
  g.mu[1] = f.mu[1];
  g.tx = FV_TX;
  g.ty = FV_TY;
  g.newton_max = kNewtonMax;
  c->max_substeps = kMaxSubsteps;
  g.ntx = (f.nx + g.tx - 1) / g.tx;
  g.nty = (f.ny + g.ty - 1) / g.ty;
  c->NP = (size_t)g.PX * g.PY;
  {
    const char *es = getenv("SIF_EXT_SWEEPS");
    c->ext_blocked = ext_blocked_ok(g) && !(es && es[0] == '1');
  }

  // one pool carved into 256-byte aligned pieces; a first pass over the
  // same carving (with a null base) measures the exact size
  size_t ncell = (size_t)f.nx * f.ny;
  // tile lists sized for the smallest supported tile (16 x 8 or 32 x 4)
  size_t ntiles = (size_t)((f.nx + 15) / 16) * ((f.ny + 3) / 4);
  char *base = nullptr;
  size_t off = 0;
  auto take = [&](size_t b) {
    char *r = base ? base + off : nullptr;
    off += (b + 255) / 256 * 256;
    return r;
  };
  auto carve = [&]() {
    auto plane = [&]() { return (double *)take(sizeof(double) * c->NP); };
    for (int k = 0; k < 2; k++)
      for (int m = 0; m < 4; m++) c->q[k][m] = plane();
    for (int k = 0; k < 2; k++)
      for (int m = 0; m < 4; m++) c->w[k][m] = plane();
    c->phi = plane();
    c->alpha = plane();
    c->ax = plane();
    c->ay = plane();
    c->sx = plane();
    c->sy = plane();
    for (int m = 0; m < 3; m++) c->xn[m] = plane();
    for (int m = 0; m < 3; m++) c->xm[m] = plane();
    for (int m = 0; m < 2; m++) c->ul[m] = plane();
    for (int k = 0; k < 2; k++)
      for (int m = 0; m < 4; m++) c->q0[k][m] = plane();
    for (int m = 0; m < 4; m++) c->prev[m] = plane();
    for (int m = 0; m < 4; m++) c->fut[m] = plane();
    for (int m = 0; m < 4; m++) c->qi[m] = plane();
    for (int m = 0; m < 3; m++) c->xc[m] = plane();
    c->phi0 = plane();
    c->phiR = plane();
    c->phia = plane();
    c->phib = plane();
    c->phie = plane();
    c->tmp = (double *)take(sizeof(double) * 16 * ncell);
    c->bandmap = (int *)take(sizeof(int) * c->NP);
    c->ext_plan = (ExtPlan *)take(sizeof(ExtPlan) * 3 * ncell);
    c->mix_plan = (MixPlan *)take(sizeof(MixPlan) * 2 * ncell);
    c->partial = (double *)take(sizeof(double) * 8 * (size_t)f.ny);
    c->integ = (double *)take(sizeof(double) * 8);
    c->band_ev = (int *)take(sizeof(int) * ncell);
    c->band_ls = (int *)take(sizeof(int) * ncell);
    c->rext_ls = (int *)take(sizeof(int) * ncell);
    c->cut = (int *)take(sizeof(int) * ncell);
    c->tiles[0] = (int *)take(sizeof(int) * ntiles);
    c->tiles[1] = (int *)take(sizeof(int) * ntiles);
    c->etiles = (int *)take(sizeof(int) * ext_tiles(c->g));
    c->nostate[0] = (unsigned char *)take(c->NP);
    c->nostate[1] = (unsigned char *)take(c->NP);
    c->sc = (Scalars *)take(sizeof(Scalars));
  };
  carve();
  size_t total = off;
  if (cudaMalloc(&c->pool, total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return SIF_ECUDA;
  }
  cudaMemset(c->pool, 0, total);
  c->band_work = (int)ncell;
  c->pool_bytes = total;
  base = (char *)c->pool;
  off = 0;
  carve();
  cudaMemset(c->bandmap, 0xff, sizeof(int) * c->NP);
  if (off != total) {
    cudaFree(c->pool);
    delete c;
    return SIF_ECUDA;
  }
  if (cudaMallocHost(&c->hsc, sizeof(Scalars)) != cudaSuccess ||
      cudaMallocHost(&c->hbuf, sizeof(double) * 16) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->pool);
    if (c->hsc) cudaFreeHost(c->hsc);
    delete c;
    return SIF_ECUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->pool);
    cudaFreeHost(c->hsc);
    cudaFreeHost(c->hbuf);
    delete c;
    return SIF_ECUDA;
  }
  const char *dbg = getenv("SIF_DEBUG_SYNC");
  c->debug_sync = dbg && dbg[0] == '1';
  snprintf(c->err, sizeof(c->err), "ok");
  *out = c;
  return SIF_OK;
}

extern "C" void sif_destroy(sif_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  free_graphs(c);
  if (c->tape_planes) cudaFree(c->tape_planes);
  if (c->adj_pool) cudaFree(c->adj_pool);
  for (int i = 0; i < 4; i++)
    if (c->cap[i]) cudaStreamDestroy(c->cap[i]);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  cudaFree(c->pool);
  cudaFreeHost(c->hsc);
  cudaFreeHost(c->hbuf);
  delete c;
}

extern "C" const char *sif_last_error(const sif_ctx *c) { return c ? c->err : "null context"; }

// ---------------------------------------------------------------------
// building blocks, in the order of the CPU reference

// opt-in fault localisation: synchronise after a phase and report the
// first failing one on stderr
static void dbg(sif_ctx *c, const char *phase) {
  if (!c->debug_sync || c->capturing) return;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) fprintf(stderr, "libsif: %s failed: %s\n", phase, cudaGetErrorString(e));
}

// record the first error of a graph-building call in c->gerr
#define GCK(call)                                  \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess && !c->gerr) c->gerr = e_; \
  } while (0)

// a captured branch pending: what is captured next depends on its tail too
static void side_join(sif_ctx *c) {
  if (!c->side_pending) return;
  c->side_pending = 0;
  GCK(cudaStreamUpdateCaptureDependencies(c->st, c->br_tail,
                                          c->br_tail_has_ed ? c->br_tail_ed : nullptr,
                                          c->br_ntail, cudaStreamAddCaptureDependencies));
}

// capture launch(), which starts from the current dependency set, as a
// branch: afterwards the capture continues from the same set, and the
// branch is joined by side_join.  Outside capture launch() just runs.
template <class F>
static void side_branch(sif_ctx *c, F launch) {
  side_join(c);
  if (!c->capturing) {
    launch();
    return;
  }
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  GCK(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, nullptr, &deps, &ed, &nd));
  if (c->gerr || nd > 8) {
    launch();  // no branch (in order)
    return;
  }
  c->br_nbase = nd;
  c->br_base_has_ed = ed != nullptr;
  for (size_t i = 0; i < nd; i++) {
    c->br_base[i] = deps[i];
    if (ed) c->br_base_ed[i] = ed[i];
  }
  launch();
  GCK(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, nullptr, &deps, &ed, &nd));
  if (c->gerr || nd > 8) return;  // the branch stays in order
  c->br_ntail = nd;
  c->br_tail_has_ed = ed != nullptr;
  for (size_t i = 0; i < nd; i++) {
    c->br_tail[i] = deps[i];
    if (ed) c->br_tail_ed[i] = ed[i];
  }
  GCK(cudaStreamUpdateCaptureDependencies(c->st, c->br_base,
                                          c->br_base_has_ed ? c->br_base_ed : nullptr,
                                          c->br_nbase, cudaStreamSetCaptureDependencies));
  if (!c->gerr) c->side_pending = 1;
}

static void ghost_phi(sif_ctx *c) {
  GhostSet gs = {{c->phi}, {0}, 1};
  launch_fill_ghost(c->g, gs, c->st);
}

static void ghost_w(sif_ctx *c, int k) {
  GhostSet gs = {{c->w[k][0], c->w[k][1], c->w[k][2], c->w[k][3]}, {0, 1, 2, 0}, 4};
  launch_fill_ghost(c->g, gs, c->st);
}

static int ncell(const sif_ctx *c) { return c->g.nx * c->g.ny; }
static int ntile(const sif_ctx *c) { return c->g.ntx * c->g.nty; }

static int band_work(const sif_ctx *c);

// level set changed: ghosts, geometry, cut list, band list and map, tile
// lists.  after_ls: phi changed by a level-set stage or reinitialisation
// since the last call (inside the band only, the interface by less than a
// cell), so only the previous band's cells can change their geometry;
// otherwise (initial data, a restored or replayed phi) the whole grid.
static void geometry(sif_ctx *c, bool after_ls = false) {
  side_join(c);  // the band list changes
  // a level-set stage and the reinitialisation write phi's ghost images
  // with its band values; anything else that sets phi needs the fill
  if (!after_ls) ghost_phi(c);
  const bool band = after_ls && c->g.band >= 3.0;
  launch_geometry(c->g, c->phi, c->alpha, c->ax, c->ay, c->sx, c->sy, c->cut, c->sc, c->st,
                  band ? c->band_ev : nullptr, band ? &c->sc->n_band : nullptr,
                  band ? band_work(c) : 0);
  launch_band_tiles(c->g, c->phi, c->band_ev, c->bandmap, c->etiles, c->tiles[0], c->tiles[1],
                    c->sc, c->st);
  dbg(c, "geometry");
}

// grids of the band kernels are sized from the last band size seen on the
// host (the kernels loop over the device count, so any size is correct)
static int band_work(const sif_ctx *c) {
  int w = c->band_work + c->band_work / 4 + 1024;
  return w < ncell(c) ? w : ncell(c);
}

// small-cell mixing of the fluids in mask (bit k = fluid k)
static void mix2(sif_ctx *c, int mask, double *const qN[4], double *const qP[4]) {
  side_join(c);
  launch_mix2(c->g, mask, qN, qP, c->alpha, c->phi, c->band_ev, c->bandmap, &c->sc->n_band,
              c->mix_plan, ncell(c), band_work(c), c->tmp, c->st);
  dbg(c, "mix");
}
static void mix_both(sif_ctx *c) { mix2(c, 3, c->q[0], c->q[1]); }
static void mix_one(sif_ctx *c, int k, double *const q[4]) {
  mix2(c, 1 << k, k == 0 ? q : nullptr, k == 1 ? q : nullptr);
}
// both fluids on the same geometry in one mixing pass: fluid 1's state q1,
// the other fluid's q2 (the fluids' mixings are independent)
static void mix_pair(sif_ctx *c, int f1, double *const q1[4], double *const q2[4]) {
  mix2(c, 3, f1 == 0 ? q1 : q2, f1 == 0 ? q2 : q1);
}

// extension plans of the three fields on the current geometry and the
// extension of both fluids' stencil states (Sec. 2.3) over the band
static void extend_states(sif_ctx *c) {
  if (c->ext_blocked) {
    launch_ext_setup(c->g, c->alpha, c->phi, c->sx, c->sy, c->band_ev, &c->sc->n_band,
                     c->bandmap, c->ext_plan, ncell(c), band_work(c), c->nostate, c->st, c->w[0],
                     c->w[1], c->tmp, 1);
    launch_ext_blocked(c->g, c->w[0], c->w[1], c->ul[0], c->ul[1], 0, 2, c->ext_plan, ncell(c),
                       c->etiles, &c->sc->n_band, c->bandmap, c->band_ev, band_work(c), c->tmp,
                       c->alpha, c->nostate, c->sc, c->num_sms, c->st);
    return;
  }
  // the plan kernel also takes the stencil states' first sweep
  const bool first = c->g.ext_iters >= 1;
  launch_ext_setup(c->g, c->alpha, c->phi, c->sx, c->sy, c->band_ev, &c->sc->n_band, c->bandmap,
                   c->ext_plan, ncell(c), band_work(c), c->nostate, c->st, c->w[0], c->w[1],
                   first ? c->tmp : nullptr);
  launch_ext_sweeps(c->g, c->w[0], c->w[1], c->ul[0], c->ul[1], 0, 2, c->ext_plan, ncell(c),
                    band_work(c), c->band_ev, &c->sc->n_band, c->tmp, c->alpha, c->nostate,
                    c->sc, c->st, first ? 1 : 0);
}

// interaction step for stage states qs of both fluids and the current phi:
// stencil states and their extension, interface Riemann problems, exchange
// flux and the level-set velocity in cut cells (whose extension over the
// band is ul_extend, run before the stage that follows).  The geometry of
// the current phi is already in place: every change of phi (level-set
// stage, reinitialisation, initial data, restored state) is followed by
// geometry() before anything else reads it.
//
// band_fluid >= 0 names a fluid whose stencil states are read only by this
// interaction step (a sub-step of the other fluid, Sec. 3.1 step 3): its
// states are recovered in the interaction band only, unless *band_flag is
// set on the device (the last sub-step, whose second stage advances it).
static void eval(sif_ctx *c, double *const qs[2][4], int band_fluid = -1,
                 const int *band_flag = nullptr) {
  side_join(c);
  launch_sched(SCHED_RESET_MAX, c->sc, 0, 0, 0, c->st);
  launch_prim2(c->g, qs[0], qs[1], c->w[0], c->w[1], c->alpha, c->tiles[0], c->tiles[1],
               ntile(c), c->nostate, c->sc, band_fluid, band_flag, c->band_ev,
               &c->sc->n_band, c->st);
  dbg(c, "prim");
  extend_states(c);
  dbg(c, "extend");
  cudaMemsetAsync(c->ul[0], 0, sizeof(double) * c->NP, c->st);
  cudaMemsetAsync(c->ul[1], 0, sizeof(double) * c->NP, c->st);
  launch_interface(c->g, c->w[0], c->w[1], c->phi, c->sx, c->sy, c->cut, band_work(c), c->xn,
                   c->xm, c->ul[0], c->ul[1], c->sc, c->st);
  dbg(c, "interface");
}

// extension of the level-set velocity set by the last interaction step
// (its plan, band and sweep buffers stay untouched until a level-set
// stage, a reinitialisation, a mixing, a geometry or the next interaction
// step, each of which joins it first), and with s > 0 the level set's RK
// stage s after it (it reads only the extended velocity and phi, which the
// finite-volume stages do not touch), and with reinit_after the step's
// reinitialisation after that.  Called just before the
// finite-volume stage that follows the interaction step: in a captured
// graph both are a branch beside that stage.
static void ul_extend(sif_ctx *c, int s = 0, const double *dtp = nullptr,
                      bool reinit_after = false) {
  side_branch(c, [&] {
    if (c->ext_blocked)
      launch_ext_blocked(c->g, c->w[0], c->w[1], c->ul[0], c->ul[1], 2, 1, c->ext_plan, ncell(c),
                         c->etiles, &c->sc->n_band, c->bandmap, c->band_ev, band_work(c), c->tmp,
                         c->alpha, c->nostate, c->sc, c->num_sms, c->st);
    else
      launch_ext_sweeps(c->g, c->w[0], c->w[1], c->ul[0], c->ul[1], 2, 1, c->ext_plan, ncell(c),
                        band_work(c), c->band_ev, &c->sc->n_band, c->tmp, c->alpha, c->nostate,
                        c->sc, c->st);
    if (s > 0)
      launch_ls_stage(c->g, s, c->cfg.rk_order, c->phi, c->phi0, c->ul[0], c->ul[1], c->band_ls,
                      &c->sc->n_band_ls, ncell(c), c->tmp, dtp, c->st);
    if (reinit_after)
      launch_reinit(c->g, c->phi, c->phiR, c->rext_ls, &c->sc->n_rext, ncell(c), c->tmp, c->st);
  });
  dbg(c, "ls_extend");
}

// evaluation of fluid 1's third stage in an RK3 cycle (at t^n + dt1/2, the
// level set interpolated there): fluid 1's stencil states recovered and
// extended on the current geometry with its wave speeds, no exchange flux
// (the correction quantities would remove that evaluation's exchange from
// fluid 1 exactly); fluid 2's stencil states are re-extended where they are
static void eval_third(sif_ctx *c, int f1) {
  side_join(c);
  launch_sched(SCHED_RESET_MAX, c->sc, 0, 0, 0, c->st);
  launch_prim2(c->g, c->q[0], c->q[1], c->w[0], c->w[1], c->alpha, c->tiles[0], c->tiles[1],
               ntile(c), c->nostate, c->sc, -1, nullptr, c->band_ev, &c->sc->n_band, c->st,
               1 - f1);
  extend_states(c);
  launch_zero_cut(c->g, c->xn, c->xm, c->cut, &c->sc->n_cut, band_work(c), c->st);
  dbg(c, "third-stage evaluation");
}

static void d2d_plane(sif_ctx *c, double *dst, const double *src) {
  cudaMemcpyAsync(dst, src, sizeof(double) * c->NP, cudaMemcpyDeviceToDevice, c->st);
}

static void copy_planes(sif_ctx *c, double *const dst[4], double *const src[4], int n) {
  for (int m = 0; m < n; m++)
    cudaMemcpyAsync(dst[m], src[m], sizeof(double) * c->NP, cudaMemcpyDeviceToDevice, c->st);
}

static void fv(sif_ctx *c, int k, int s, double *const dst[4], double *const base[4],
               double *const cur[4], const double *dtp) {
  // the exchange flux planes of fluid k (fluid P's negated)
  double *const *X = k == 0 ? c->xn : c->xm;
  ghost_w(c, k);
  launch_fv_stage(c->g, k, s, c->cfg.rk_order, dst, base, cur, c->w[k], c->ax, c->ay, c->sx,
                  c->sy, X[0], X[1], X[2], c->tiles[k], ntile(c), c->num_sms, dtp,
                  c->sc, c->st);
  if (c->g.mu[k] > 0.0)
    launch_viscous(c->g, k, s, c->cfg.rk_order, dst, c->w[k], c->ax, c->ay, c->tiles[k], ntile(c),
                   dtp, c->sc, c->st);
  dbg(c, "fv_stage");
}

// start of a level-set RK step: keep phi^n and fix the step's band (and
// its face-neighbour extension for the reinitialisation) from it
static void ls_begin(sif_ctx *c) {
  cudaMemcpyAsync(c->phi0, c->phi, sizeof(double) * c->NP, cudaMemcpyDeviceToDevice, c->st);
  launch_band_lists(c->g, c->phi, c->band_ls, c->rext_ls, &c->sc->n_band_ls, c->st);
}

// where a recorded step keeps its level set after stage 1 and the
// Lax-Friedrichs speeds of stage 2
struct TapeHook {
  double *phi1;
  double *lf2;
  double *W[2][2][4];          // stage, fluid, component
  unsigned char *flags2[2];    // stage 2, fluid
};

// one RK step of both fluids and the level set, the first interaction
// step having been evaluated; dtp points to the step size on the device
static void single_step_after_eval(sif_ctx *c, const double *dtp, const TapeHook *rec = nullptr) {
  int S = c->cfg.rk_order;
  for (int k = 0; k < 2; k++) copy_planes(c, c->q0[k], c->q[k], 4);
  ls_begin(c);
  for (int s = 1; s <= S; s++) {
    if (s > 1) eval(c, c->q);
    ul_extend(c, s, dtp, s == S);
    if (rec && s == 2) {
      cudaMemcpyAsync(rec->lf2, c->sc->lf, sizeof(c->sc->lf), cudaMemcpyDeviceToDevice, c->st);
      for (int k = 0; k < 2; k++)
        cudaMemcpyAsync(rec->flags2[k], c->nostate[k], c->NP, cudaMemcpyDeviceToDevice, c->st);
    }
    for (int k = 0; k < 2; k++) fv(c, k, s, c->q[k], c->q0[k], c->q[k], dtp);
    if (rec && s <= 2)
      for (int k = 0; k < 2; k++)
        for (int m = 0; m < 4; m++)
          cudaMemcpyAsync(rec->W[s - 1][k][m], c->w[k][m], sizeof(double) * c->NP,
                          cudaMemcpyDeviceToDevice, c->st);
    if (rec && s == 1) {
      side_join(c);  // the level set's first stage
      cudaMemcpyAsync(rec->phi1, c->phi, sizeof(double) * c->NP, cudaMemcpyDeviceToDevice, c->st);
    }
    geometry(c, true);
    mix_both(c);
  }
}

// update counters at the start of a call: active-tile and open-cell stage updates
struct Upd {
  unsigned long long tile, open;
};

static int finish(sif_ctx *c, sif_cycle_info *info, Upd upd0) {
  side_join(c);
  int rc = check_launch(c, "step");
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->band_work = c->hsc->n_band;
  if (info) {
    info->t = c->hsc->t;
    info->cell_updates = (long long)(c->hsc->updates - upd0.tile);
    info->open_updates = (long long)(c->hsc->open_updates - upd0.open);
  }
  if (c->hsc->err & DERR_NONPHYS) {
    set_err(c, "non-physical state (rho <= 0 or p + p_inf <= 0) in a real cell");
    return SIF_ENONPHYS;
  }
  if (c->hsc->err & DERR_NOCONV) {
    set_err(c, "interface Riemann Newton iteration did not converge in %d iterations",
            c->g.newton_max);
    return SIF_ENOCONV;
  }
  if (c->hsc->err & DERR_TIMEOUT) {
    set_err(c, "the cycle needed more than %d fluid-2 sub-steps (state undefined)",
            c->max_substeps);
    return SIF_ETIMEOUT;
  }
  return SIF_OK;
}

static int begin_call(sif_ctx *c, double t_end, Upd *upd0) {
  if (!c->inited) {
    set_err(c, "state not initialised");
    return SIF_ESTATE;
  }
  cudaSetDevice(c->cfg.device);
  side_join(c);
  CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  upd0->tile = c->hsc->updates;
  upd0->open = c->hsc->open_updates;
  // reset the error word; set t_end
  c->hbuf[0] = t_end;
  CK(cudaMemsetAsync(&c->sc->err, 0, sizeof(int), c->st));
  CK(cudaMemcpyAsync(&c->sc->t_end, c->hbuf, sizeof(double), cudaMemcpyHostToDevice, c->st));
  return SIF_OK;
}

static void taped_step(sif_ctx *c);

extern "C" int sif_step_single_dt(sif_ctx *c, int nsteps, double t_end, sif_cycle_info *info) {
  if (!c || nsteps < 0) return SIF_EINVAL;
  if (c->tape_cap > 0 && c->tape_len + nsteps > c->tape_cap) {
    set_err(c, "adjoint tape full (%d of %d steps recorded)", c->tape_len, c->tape_cap);
    return SIF_EINVAL;
  }
  Upd upd0;
  int rc = begin_call(c, t_end, &upd0);
  if (rc) return rc;
  for (int n = 0; n < nsteps; n++) {
    if (t_end > 0.0) {
      // the host needs the time to stop at t_end
      CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (c->hsc->t >= t_end) break;
    }
    if (c->tape_cap > 0) {
      taped_step(c);  // the same kernels in the same order, recording
    } else if (ensure_graphs(c) == SIF_OK) {
      CK(cudaGraphLaunch(c->g_single, c->st));
    } else if (c->require_graphs && c->use_graphs == 0 && !c->no_graph_env) {
      return SIF_ECUDA;
    } else {
      eval(c, c->q);
      launch_sched(SCHED_SINGLE_DT, c->sc, c->g.cfl, 0, 0, c->st);
      single_step_after_eval(c, &c->sc->dt);
      launch_sched(SCHED_T_SINGLE, c->sc, 0, 0, 0, c->st);
    }
  }
  rc = finish(c, info, upd0);
  if (info) {
    info->dt1 = info->dt2 = c->hsc->dt;
    info->n_raw = info->n_used = 1.0;
    info->role_fluid1 = -1;
    info->substeps = 1;
  }
  return rc;
}

static int read_scalars(sif_ctx *c) {
  side_join(c);
  CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->band_work = c->hsc->n_band;
  return SIF_OK;
}

static void third_stage(sif_ctx *c, int f1);

// one RK3 cycle with fluid 1 = f1 issued from the host: the kernels of
// graph_substep3 / graph_cycle_body3 in the same order, the branches
// taken on the host after reading the scheduler's decisions
static int cycle3(sif_ctx *c, int f1, sif_cycle_info *info) {
  const int f2 = 1 - f1;
  const double cfl = c->g.cfl, thr = c->cfg.ratio_threshold;
  const double b12 = 1.0 / 6.0, b3 = 2.0 / 3.0;
  for (int m = 0; m < 3; m++) cudaMemsetAsync(c->xc[m], 0, sizeof(double) * c->NP, c->st);
  copy_planes(c, c->prev, c->q[f1], 4);
  copy_planes(c, c->fut, c->q[f1], 4);
  fv(c, f1, 1, c->fut, c->prev, c->prev, &c->sc->dt1);
  double *qs[2][4];
  for (int m = 0; m < 4; m++) {
    qs[f1][m] = c->qi[m];
    qs[f2][m] = c->q[f2][m];
  }
  int sub = 0;
  for (;;) {
    sub++;
    if (sub > 1) {
      launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                    band_work(c), c->st);
      mix_one(c, f1, c->qi);
      eval(c, qs, f1);
      launch_sched(SCHED_SUBSTEP, c->sc, cfl, thr, 0, c->st);
    } else {
      launch_sched(SCHED_FIRST_SUB, c->sc, cfl, thr, 0, c->st);
    }
    int rc = read_scalars(c);
    if (rc) return rc;
    if (c->hsc->err || !(c->hsc->dt2 > 0.0) || !(c->hsc->dt2 < 1e300)) {
      if (!c->hsc->err) set_err(c, "fluid-2 time step is not positive and finite");
      return c->hsc->err ? SIF_OK : SIF_ENONPHYS;
    }
    const int last = c->hsc->last, single = c->hsc->single;
    launch_record(c->g, sub == 1, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1],
                  c->xc[2], c->sc, c->st, b12, 1);
    launch_copy_if(&c->sc->snap_a, c->phi, c->phia, c->NP, c->st);
    copy_planes(c, c->q0[f2], c->q[f2], 4);
    ls_begin(c);
    ul_extend(c, 1, &c->sc->dt2);
    fv(c, f2, 1, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
    geometry(c, true);
    if (last) {
      mix_pair(c, f1, c->fut, c->q[f2]);
      copy_planes(c, c->qi, c->fut, 4);
    } else {
      launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                    band_work(c), c->st);
      mix_pair(c, f1, c->qi, c->q[f2]);
    }
    eval(c, qs, last ? -1 : f1);
    ul_extend(c, 2, &c->sc->dt2);
    launch_record(c->g, last, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1], c->xc[2],
                  c->sc, c->st, b12, 1);
    fv(c, f2, 2, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
    if (last) fv(c, f1, 2, c->q[f1], c->prev, c->fut, &c->sc->dt1);
    geometry(c, true);
    if (single) {
      mix_pair(c, f1, c->q[f1], c->q[f2]);
      copy_planes(c, c->qi, c->q[f1], 4);
    } else {
      mix_one(c, f2, c->q[f2]);
      launch_sched(SCHED_THETA3, c->sc, 0, 0, 0, c->st);
      launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                    band_work(c), c->st);
      mix_one(c, f1, c->qi);
    }
    eval(c, qs, single ? -1 : f1);
    ul_extend(c, 3, &c->sc->dt2, true);
    launch_record(c->g, single, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1], c->xc[2],
                  c->sc, c->st, b3, 1);
    fv(c, f2, 3, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
    if (single) fv(c, f1, 3, c->q[f1], c->prev, c->q[f1], &c->sc->dt1);
    geometry(c, true);
    mix_one(c, f2, c->q[f2]);
    launch_sched(SCHED_SNAPB, c->sc, 0, 0, 0, c->st);
    launch_copy_if(&c->sc->snap_b, c->phi, c->phib, c->NP, c->st);
    if (last) break;
    launch_sched(SCHED_ADVANCE, c->sc, cfl, thr, 0, c->st);
    if (sub >= c->max_substeps) {
      set_err(c, "the cycle needed more than %d fluid-2 sub-steps (state undefined)",
              c->max_substeps);
      return SIF_ETIMEOUT;
    }
  }
  if (sub > 1) third_stage(c, f1);
  if (c->cfg.flux_correction) launch_correction(c->g, c->q[f1], c->xc[0], c->xc[1], c->xc[2], c->st);
  mix_one(c, f1, c->q[f1]);
  launch_sched(SCHED_T_CYCLE, c->sc, 0, 0, 0, c->st);
  if (info) info->substeps = sub;
  return SIF_OK;
}

// one cycle of the accelerated method (Sec. 3.1 steps 1-5)
static int cycle(sif_ctx *c, sif_cycle_info *info) {
  const double cfl = c->g.cfl, thr = c->cfg.ratio_threshold;
  eval(c, c->q);
  launch_sched(SCHED_CYCLE_BEGIN, c->sc, cfl, thr, c->cfg.force_ratio_one, c->st);
  int rc = read_scalars(c);
  if (rc) return rc;
  if (info) {
    info->n_raw = c->hsc->n_raw;
    info->role_fluid1 = c->hsc->f1;
  }
  if (c->hsc->mode == 0) {
    single_step_after_eval(c, &c->sc->dt);
    launch_sched(SCHED_T_SINGLE, c->sc, 0, 0, 0, c->st);
    if (info) {
      info->dt1 = info->dt2 = c->hsc->dt;
      info->n_used = 1.0;
      info->substeps = 1;
    }
    return SIF_OK;
  }
  const int f1 = c->hsc->f1, f2 = 1 - f1;
  if (info) {
    info->dt1 = c->hsc->dt1;
    info->dt2 = c->hsc->dt2;
    info->n_used = c->hsc->n_used;
  }
  if (c->cfg.rk_order == 3) return cycle3(c, f1, info);
  for (int m = 0; m < 3; m++) cudaMemsetAsync(c->xc[m], 0, sizeof(double) * c->NP, c->st);
  // step 2: fluid-1 first RK stage with dt1; previous and future states
  copy_planes(c, c->prev, c->q[f1], 4);
  // the stage writes fluid 1's tiles only; elsewhere the future state is
  // the state itself (no open face, no exchange)
  copy_planes(c, c->fut, c->q[f1], 4);
  fv(c, f1, 1, c->fut, c->prev, c->prev, &c->sc->dt1);
  double *qs[2][4];
  int sub = 0;
  for (;;) {
    sub++;
    if (sub > 1) {
      launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
      mix_one(c, f1, c->qi);
      for (int m = 0; m < 4; m++) {
        qs[f1][m] = c->qi[m];
        qs[f2][m] = c->q[f2][m];
      }
      eval(c, qs, f1);
      launch_sched(SCHED_SUBSTEP, c->sc, cfl, thr, 0, c->st);
    } else {
      launch_sched(SCHED_FIRST_SUB, c->sc, cfl, thr, 0, c->st);
    }
    rc = read_scalars(c);
    if (rc) return rc;
    if (c->hsc->err || !(c->hsc->dt2 > 0.0) || !(c->hsc->dt2 < 1e300)) {
      // a failed interaction step leaves no usable fluid-2 step: stop here
      // and let the caller see the device error word
      if (!c->hsc->err) set_err(c, "fluid-2 time step is not positive and finite");
      return c->hsc->err ? SIF_OK : SIF_ENONPHYS;
    }
    const int last = c->hsc->last;
    launch_record(c->g, sub == 1, c->cut, ncell(c), c->xn, c->xm, c->xc[0],
                  c->xc[1], c->xc[2], c->sc, c->st);
    // step 3: fluid-2 and level-set first RK stage with dt2
    copy_planes(c, c->q0[f2], c->q[f2], 4);
    ls_begin(c);
    ul_extend(c, 1, &c->sc->dt2);  // of the cycle's first or this sub-step's interaction step
    fv(c, f2, 1, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
    geometry(c, true);
    if (last) {
      mix_pair(c, f1, c->fut, c->q[f2]);
      for (int m = 0; m < 4; m++) qs[f1][m] = c->fut[m];
    } else {
      launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
      mix_pair(c, f1, c->qi, c->q[f2]);
      for (int m = 0; m < 4; m++) qs[f1][m] = c->qi[m];
    }
    for (int m = 0; m < 4; m++) qs[f2][m] = c->q[f2][m];
    eval(c, qs, last ? -1 : f1);
    ul_extend(c, 2, &c->sc->dt2, true);
    launch_record(c->g, last, c->cut, ncell(c), c->xn, c->xm, c->xc[0],
                  c->xc[1], c->xc[2], c->sc, c->st);
    // step 4 (and 5 on the last sub-step): second RK stage
    fv(c, f2, 2, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
    if (last) fv(c, f1, 2, c->q[f1], c->prev, c->fut, &c->sc->dt1);
    if (last) {
      if (c->cfg.flux_correction) launch_correction(c->g, c->q[f1], c->xc[0], c->xc[1], c->xc[2], c->st);
      geometry(c, true);
      mix_both(c);
      break;
    }
    launch_sched(SCHED_ADVANCE, c->sc, cfl, thr, 0, c->st);
    geometry(c, true);
    mix_one(c, f2, c->q[f2]);
    if (sub >= c->max_substeps) {
      set_err(c, "the cycle needed more than %d fluid-2 sub-steps (state undefined)",
              c->max_substeps);
      return SIF_ETIMEOUT;
    }
  }
  launch_sched(SCHED_T_CYCLE, c->sc, 0, 0, 0, c->st);
  if (info) info->substeps = sub;
  return SIF_OK;
}

// ---------------------------------------------------------------------
// device-driven graphs: one CUDA graph runs a whole accelerated cycle;
// conditional IF nodes follow the scheduler's decisions (single step or
// cycle, fluid 1's identity, first and last sub-step) and a WHILE node
// repeats the fluid-2 sub-step, so no host round trip remains inside a
// cycle.  The kernels are exactly those of the host-driven path.

static cudaGraph_t capture_graph(sif_ctx *c) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  GCK(cudaStreamGetCaptureInfo(c->st, &st, nullptr, &g, nullptr, nullptr, nullptr));
  return g;
}

static cudaGraphConditionalHandle new_handle(sif_ctx *c) {
  cudaGraphConditionalHandle h = 0;
  GCK(cudaGraphConditionalHandleCreate(&h, capture_graph(c), 0, cudaGraphCondAssignDefault));
  return h;
}

// append a conditional node to the graph being captured on c->st and
// capture `body` into its body graph on the next capture stream
template <class F>
static void cond_node(sif_ctx *c, cudaGraphConditionalHandle h, bool loop, F body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  side_join(c);  // a pending branch joins before a conditional node
  GCK(cudaStreamGetCaptureInfo(c->st, &st, nullptr, &g, &deps, &ed, &nd));
  if (c->gerr) return;
  // the parameter union has no default constructor: zeroed raw storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(raw);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = loop ? cudaGraphCondTypeWhile : cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  GCK(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
  if (c->gerr) return;
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  GCK(cudaStreamUpdateCaptureDependencies(c->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  if (c->cap_depth >= 3) {
    c->gerr = cudaErrorNotSupported;
    return;
  }
  cudaStream_t outer = c->st, inner = c->cap[++c->cap_depth];
  GCK(cudaStreamBeginCaptureToGraph(inner, bodyg, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal));
  c->st = inner;
  if (!c->gerr) body();
  side_join(c);
  c->st = outer;
  cudaGraph_t out = nullptr;
  GCK(cudaStreamEndCapture(inner, &out));
  c->cap_depth--;
}

static void copy4(sif_ctx *c, double *const dst[4], double *const src[4]) { copy_planes(c, dst, src, 4); }

// one fluid-2 sub-step of the cycle with fluid 1 = f1 (the body of the
// sub-cycle loop); hloop is the loop's condition
static void graph_substep(sif_ctx *c, int f1, cudaGraphConditionalHandle hloop) {
  const int f2 = 1 - f1;
  const double cfl = c->g.cfl, thr = c->cfg.ratio_threshold;
  double *qs[2][4];
  for (int m = 0; m < 4; m++) {
    qs[f1][m] = c->qi[m];
    qs[f2][m] = c->q[f2][m];
  }
  // after the first sub-step: fluid 1 at t2 (Eq. 7), interaction, fluid-2 step
  cudaGraphConditionalHandle hnf = new_handle(c);
  launch_cond(COND_NOT_FIRST, c->sc, hnf, 0, 0, 0, c->st);
  cond_node(c, hnf, false, [&] {
    launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
    mix_one(c, f1, c->qi);
    eval(c, qs, f1);
    launch_sched(SCHED_DT2, c->sc, cfl, thr, 0, c->st);
  });
  launch_sched(SCHED_LAST, c->sc, cfl, thr, 0, c->st);
  cudaGraphConditionalHandle hl1 = new_handle(c), hn1 = new_handle(c);
  cudaGraphConditionalHandle hl2 = new_handle(c), hn2 = new_handle(c);
  cudaGraphConditionalHandle hl3 = new_handle(c);
  launch_cond(COND_LAST, c->sc, hl1, hn1, 0, 0, c->st);
  launch_cond(COND_LAST, c->sc, hl2, hn2, 0, 0, c->st);
  launch_cond(COND_LAST_ONLY, c->sc, hl3, 0, 0, 0, c->st);
  launch_record(c->g, -1, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1],
                c->xc[2], c->sc, c->st);
  // step 3: fluid-2 and level-set first RK stage with dt2
  copy4(c, c->q0[f2], c->q[f2]);
  ls_begin(c);
  ul_extend(c, 1, &c->sc->dt2);  // of the cycle's first or this sub-step's interaction step
  fv(c, f2, 1, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
  geometry(c, true);
  cond_node(c, hl1, false, [&] {
    mix_pair(c, f1, c->fut, c->q[f2]);
    copy4(c, c->qi, c->fut);
  });
  cond_node(c, hn1, false, [&] {
    launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
    mix_pair(c, f1, c->qi, c->q[f2]);
  });
  eval(c, qs, f1, &c->sc->last);
  ul_extend(c, 2, &c->sc->dt2, true);
  launch_record(c->g, -2, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1],
                c->xc[2], c->sc, c->st);
  // step 4 (and 5 on the last sub-step): second RK stage
  fv(c, f2, 2, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
  cond_node(c, hl2, false, [&] { fv(c, f1, 2, c->q[f1], c->prev, c->fut, &c->sc->dt1); });
  cond_node(c, hl3, false, [&] {
    if (c->cfg.flux_correction)
      launch_correction(c->g, c->q[f1], c->xc[0], c->xc[1], c->xc[2], c->st);
    geometry(c, true);
    mix_both(c);
  });
  cond_node(c, hn2, false, [&] {
    launch_sched(SCHED_ADVANCE, c->sc, cfl, thr, 0, c->st);
    geometry(c, true);
    mix_one(c, f2, c->q[f2]);
  });
  launch_cond(COND_LOOP, c->sc, hloop, 0, 0, c->max_substeps, c->st);
}

static void graph_cycle_body(sif_ctx *c, int f1) {
  for (int m = 0; m < 3; m++) cudaMemsetAsync(c->xc[m], 0, sizeof(double) * c->NP, c->st);
  // step 2: fluid-1 first RK stage with dt1; previous and future states
  copy4(c, c->prev, c->q[f1]);
  // the stage writes fluid 1's tiles only; elsewhere the future state is
  // the state itself (no open face, no exchange)
  copy4(c, c->fut, c->q[f1]);
  fv(c, f1, 1, c->fut, c->prev, c->prev, &c->sc->dt1);
  cudaGraphConditionalHandle hloop = new_handle(c);
  launch_cond(COND_LOOP, c->sc, hloop, 0, 0, c->max_substeps, c->st);  // last = 0 here
  cond_node(c, hloop, true, [&] { graph_substep(c, f1, hloop); });
  launch_sched(SCHED_T_CYCLE, c->sc, 0, 0, 0, c->st);
}

// one fluid-2 sub-step of an RK3 cycle (SSP-RK3: stage evaluations at t2,
// t2 + dt2 and t2 + dt2/2, weights 1/6, 1/6, 2/3): fluid 1 by Eq. 7 at each
// evaluation, except at t1 (its future state, the evaluation shared with
// its second stage) and, when the cycle has a single sub-step, at the third
// evaluation (its own second-stage state, shared with its third stage).
// The level sets at the two sub-step boundaries around t^n + dt1/2 are
// kept for fluid 1's third stage after the loop.
static void graph_substep3(sif_ctx *c, int f1, cudaGraphConditionalHandle hloop) {
  const int f2 = 1 - f1;
  const double cfl = c->g.cfl, thr = c->cfg.ratio_threshold;
  const double b12 = 1.0 / 6.0, b3 = 2.0 / 3.0;
  double *qs[2][4];
  for (int m = 0; m < 4; m++) {
    qs[f1][m] = c->qi[m];
    qs[f2][m] = c->q[f2][m];
  }
  cudaGraphConditionalHandle hnf = new_handle(c);
  launch_cond(COND_NOT_FIRST, c->sc, hnf, 0, 0, 0, c->st);
  cond_node(c, hnf, false, [&] {
    launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
    mix_one(c, f1, c->qi);
    eval(c, qs, f1);
    launch_sched(SCHED_DT2, c->sc, cfl, thr, 0, c->st);
  });
  launch_sched(SCHED_LAST, c->sc, cfl, thr, 0, c->st);
  cudaGraphConditionalHandle hl1 = new_handle(c), hn1 = new_handle(c);
  cudaGraphConditionalHandle hl2 = new_handle(c), hn3 = new_handle(c);
  cudaGraphConditionalHandle hs1 = new_handle(c), hns1 = new_handle(c);
  cudaGraphConditionalHandle hs2 = new_handle(c);
  launch_cond(COND_LAST, c->sc, hl1, hn1, 0, 0, c->st);
  launch_cond(COND_LAST, c->sc, hl2, hn3, 0, 0, c->st);
  launch_cond(COND_SINGLE, c->sc, hs1, hns1, 0, 0, c->st);
  launch_cond(COND_SINGLE_ONLY, c->sc, hs2, 0, 0, 0, c->st);
  launch_record(c->g, -1, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1], c->xc[2], c->sc,
                c->st, b12, 1);
  launch_copy_if(&c->sc->snap_a, c->phi, c->phia, c->NP, c->st);
  // stage 1 of fluid 2 and the level set
  copy4(c, c->q0[f2], c->q[f2]);
  ls_begin(c);
  ul_extend(c, 1, &c->sc->dt2);
  fv(c, f2, 1, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
  geometry(c, true);
  // stage 2 at t2 + dt2 (at t1 on the last sub-step)
  cond_node(c, hl1, false, [&] {
    mix_pair(c, f1, c->fut, c->q[f2]);
    copy4(c, c->qi, c->fut);
  });
  cond_node(c, hn1, false, [&] {
    launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
    mix_pair(c, f1, c->qi, c->q[f2]);
  });
  eval(c, qs, f1, &c->sc->last);
  ul_extend(c, 2, &c->sc->dt2);
  launch_record(c->g, -2, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1], c->xc[2], c->sc,
                c->st, b12, 1);
  fv(c, f2, 2, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
  cond_node(c, hl2, false, [&] { fv(c, f1, 2, c->q[f1], c->prev, c->fut, &c->sc->dt1); });
  geometry(c, true);
  // stage 3 at t2 + dt2/2
  cond_node(c, hs1, false, [&] {
    mix_pair(c, f1, c->q[f1], c->q[f2]);
    copy4(c, c->qi, c->q[f1]);
  });
  cond_node(c, hns1, false, [&] {
    mix_one(c, f2, c->q[f2]);
    launch_sched(SCHED_THETA3, c->sc, 0, 0, 0, c->st);
    launch_interp(c->g, c->qi, c->prev, c->fut, &c->sc->theta, c->band_ev, &c->sc->n_band,
                  band_work(c), c->st);
    mix_one(c, f1, c->qi);
  });
  eval(c, qs, f1, &c->sc->single);
  ul_extend(c, 3, &c->sc->dt2, true);
  launch_record(c->g, -3, c->cut, ncell(c), c->xn, c->xm, c->xc[0], c->xc[1], c->xc[2], c->sc,
                c->st, b3, 1);
  fv(c, f2, 3, c->q[f2], c->q0[f2], c->q[f2], &c->sc->dt2);
  cond_node(c, hs2, false, [&] { fv(c, f1, 3, c->q[f1], c->prev, c->q[f1], &c->sc->dt1); });
  geometry(c, true);
  mix_one(c, f2, c->q[f2]);
  launch_sched(SCHED_SNAPB, c->sc, 0, 0, 0, c->st);
  launch_copy_if(&c->sc->snap_b, c->phi, c->phib, c->NP, c->st);
  cond_node(c, hn3, false, [&] { launch_sched(SCHED_ADVANCE, c->sc, cfl, thr, 0, c->st); });
  launch_cond(COND_LOOP, c->sc, hloop, 0, 0, c->max_substeps, c->st);
}

// fluid 1's third RK3 stage at t^n + dt1/2 on the level set interpolated
// between the kept ones (a fluid-1-only evaluation, see eval_third); the
// level set of the cycle's end is restored afterwards
static void third_stage(sif_ctx *c, int f1) {
  d2d_plane(c, c->phie, c->phi);
  launch_sched(SCHED_W3, c->sc, 0, 0, 0, c->st);
  launch_phi_interp(c->g, c->phi, c->phia, c->phib, &c->sc->theta, c->st);
  ghost_phi(c);
  geometry(c, true);
  mix_one(c, f1, c->q[f1]);
  eval_third(c, f1);
  fv(c, f1, 3, c->q[f1], c->prev, c->q[f1], &c->sc->dt1);
  d2d_plane(c, c->phi, c->phie);
  geometry(c, true);
}

static void graph_cycle_body3(sif_ctx *c, int f1) {
  for (int m = 0; m < 3; m++) cudaMemsetAsync(c->xc[m], 0, sizeof(double) * c->NP, c->st);
  copy4(c, c->prev, c->q[f1]);
  copy4(c, c->fut, c->q[f1]);
  fv(c, f1, 1, c->fut, c->prev, c->prev, &c->sc->dt1);
  cudaGraphConditionalHandle hloop = new_handle(c);
  launch_cond(COND_LOOP, c->sc, hloop, 0, 0, c->max_substeps, c->st);
  cond_node(c, hloop, true, [&] { graph_substep3(c, f1, hloop); });
  // more than one sub-step: fluid 1's third stage after the loop (every
  // handle created in a graph gets its conditional node)
  cudaGraphConditionalHandle hns = new_handle(c);
  launch_cond(COND_MULTI_ONLY, c->sc, hns, 0, 0, 0, c->st);
  cond_node(c, hns, false, [&] { third_stage(c, f1); });
  if (c->cfg.flux_correction)
    launch_correction(c->g, c->q[f1], c->xc[0], c->xc[1], c->xc[2], c->st);
  mix_one(c, f1, c->q[f1]);
  launch_sched(SCHED_T_CYCLE, c->sc, 0, 0, 0, c->st);
}

// one accelerated cycle, captured onto c->st (which must be capturing)
static void capture_cycle(sif_ctx *c) {
  const double cfl = c->g.cfl, thr = c->cfg.ratio_threshold;
  cudaGraphConditionalHandle hs = new_handle(c), h0 = new_handle(c), h1 = new_handle(c);
  eval(c, c->q);
  launch_sched(SCHED_CYCLE_BEGIN, c->sc, cfl, thr, c->cfg.force_ratio_one, c->st);
  launch_cond(COND_CYCLE, c->sc, hs, h0, h1, 0, c->st);
  cond_node(c, hs, false, [&] {
    single_step_after_eval(c, &c->sc->dt);
    launch_sched(SCHED_T_SINGLE, c->sc, 0, 0, 0, c->st);
  });
  if (c->cfg.rk_order == 3) {
    cond_node(c, h0, false, [&] { graph_cycle_body3(c, 0); });
    cond_node(c, h1, false, [&] { graph_cycle_body3(c, 1); });
  } else {
    cond_node(c, h0, false, [&] { graph_cycle_body(c, 0); });
    cond_node(c, h1, false, [&] { graph_cycle_body(c, 1); });
  }
}

static void free_graphs(sif_ctx *c) {
  if (c->g_cycle) cudaGraphExecDestroy(c->g_cycle);
  if (c->g_single) cudaGraphExecDestroy(c->g_single);
  if (c->g_cycle_tmpl) cudaGraphDestroy(c->g_cycle_tmpl);
  c->g_cycle = c->g_single = nullptr;
  c->g_cycle_tmpl = nullptr;
  c->graph_gen++;
}

static int bucket_for(int n) {
  int b = 1024;
  while (b < n + n / 2 + 1024) b *= 2;
  return b;
}

static int build_graphs(sif_ctx *c) {
  free_graphs(c);
  c->graph_bucket = bucket_for(c->band_work);
  int saved_work = c->band_work;
  c->band_work = c->graph_bucket;  // grids of the band kernels in the graphs
  c->gerr = 0;
  c->capturing = 1;
  c->cap_depth = 0;
  cudaGraph_t gc = nullptr, gs = nullptr;
  const double cfl = c->g.cfl;
  // accelerated cycle
  GCK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  if (!c->gerr) capture_cycle(c);
  side_join(c);
  cudaError_t e = cudaStreamEndCapture(c->st, &gc);
  if (!c->gerr && e != cudaSuccess) c->gerr = e;
  // original single-time-step method
  if (!c->gerr) {
    GCK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    eval(c, c->q);
    launch_sched(SCHED_SINGLE_DT, c->sc, cfl, 0, 0, c->st);
    single_step_after_eval(c, &c->sc->dt);
    launch_sched(SCHED_T_SINGLE, c->sc, 0, 0, 0, c->st);
    side_join(c);
    e = cudaStreamEndCapture(c->st, &gs);
    if (!c->gerr && e != cudaSuccess) c->gerr = e;
  }
  c->capturing = 0;
  c->band_work = saved_work;
  if (!c->gerr && gc) GCK(cudaGraphInstantiate(&c->g_cycle, gc, 0));
  if (!c->gerr && gs) GCK(cudaGraphInstantiate(&c->g_single, gs, 0));
  if (gc && !c->gerr) c->g_cycle_tmpl = gc;
  else if (gc) cudaGraphDestroy(gc);
  if (gs) cudaGraphDestroy(gs);
  cudaGetLastError();
  if (c->gerr) {
    set_err(c, "cycle graph capture failed (%s); cycles are issued from the host",
            cudaGetErrorString((cudaError_t)c->gerr));
    free_graphs(c);
    c->use_graphs = 0;  // fall back to the host-driven sequence
    return SIF_ECUDA;
  }
  return SIF_OK;
}

// 0: graphs in use; SIF_ECUDA: the host issues the kernels instead (graphs
// switched off by SIF_NO_GRAPH=1 or a failed capture, whose reason is in
// c->err).  With SIF_REQUIRE_GRAPHS=1 a step call returns that failure.
static int ensure_graphs(sif_ctx *c) {
  if (!c->use_graphs) return SIF_ECUDA;
  // rebuild when the band outgrew the baked grid sizes or shrank far below
  int want = bucket_for(c->band_work);
  if (c->g_cycle && c->g_single && want <= c->graph_bucket && c->graph_bucket <= 4 * want)
    return SIF_OK;
  return build_graphs(c);
}

extern "C" int sif_step_multi_dt(sif_ctx *c, int ncycles, double t_end, sif_cycle_info *info) {
  if (!c || ncycles < 0) return SIF_EINVAL;
  if (c->tape_cap > 0) {
    set_err(c, "the adjoint tape records single-time-step steps only");
    return SIF_ESTATE;
  }
  Upd upd0;
  int rc = begin_call(c, t_end, &upd0);
  if (rc) return rc;
  const int graphs = ensure_graphs(c);
  if (graphs != SIF_OK && c->require_graphs && !c->no_graph_env) return SIF_ECUDA;
  if (graphs == SIF_OK) {
    for (int n = 0; n < ncycles; n++) {
      if (t_end > 0.0) {
        rc = read_scalars(c);
        if (rc) return rc;
        if (c->hsc->t >= t_end || c->hsc->err) break;
      }
      CK(cudaGraphLaunch(c->g_cycle, c->st));
    }
    rc = finish(c, info, upd0);
    if (info) {
      const Scalars *h = c->hsc;
      info->role_fluid1 = h->f1;
      info->n_raw = h->n_raw;
      info->n_used = h->mode == 0 ? 1.0 : h->n_used;
      info->dt1 = h->mode == 0 ? h->dt : h->dt1;
      info->dt2 = h->mode == 0 ? h->dt : h->dt2_first;
      info->substeps = h->mode == 0 ? 1 : h->sub;
    }
    return rc;
  }
  for (int n = 0; n < ncycles; n++) {
    rc = read_scalars(c);
    if (rc) return rc;
    if (t_end > 0.0 && c->hsc->t >= t_end) break;
    rc = cycle(c, info);
    if (rc) return rc;
    if (c->hsc->err) break;
  }
  return finish(c, info, upd0);
}

// ---------------------------------------------------------------------
// state in and out

static cudaMemcpyKind kind_in(int mem) {
  return mem == SIF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind kind_out(int mem) {
  return mem == SIF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

static int put_plane(sif_ctx *c, double *dst, const double *src, int mem) {
  const Grid &g = c->g;
  CK(cudaMemcpy2DAsync(dst + gidx(g, 0, 0), sizeof(double) * g.PX, src, sizeof(double) * g.nx,
                       sizeof(double) * g.nx, g.ny, kind_in(mem), c->st));
  return SIF_OK;
}

static int get_plane(sif_ctx *c, double *dst, const double *src, int mem) {
  const Grid &g = c->g;
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * g.nx, src + gidx(g, 0, 0), sizeof(double) * g.PX,
                       sizeof(double) * g.nx, g.ny, kind_out(mem), c->st));
  return SIF_OK;
}

extern "C" int sif_init_fluids(sif_ctx *c, const double *phi, const double *pN, const double *pP,
                               int mem) {
  if (!c || !phi || !pN || !pP || (mem != SIF_HOST && mem != SIF_DEVICE)) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  size_t n = (size_t)ncell(c);
  int rc = put_plane(c, c->phi, phi, mem);
  for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, c->w[0][m], pN + m * n, mem);
  for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, c->w[1][m], pP + m * n, mem);
  if (rc) return rc;
  // scalars first: the geometry below fills the list counts in them
  CK(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), c->st));
  geometry(c);
  launch_init_state(c->g, c->q[0], c->q[1], c->w[0], c->w[1], c->alpha, c->st);
  mix_both(c);
  CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
  rc = check_launch(c, "init");
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  c->band_work = c->hsc->n_band;
  c->inited = 1;
  return SIF_OK;
}

extern "C" int sif_get_state(sif_ctx *c, double *qN, double *qP, double *phi, int mem) {
  if (!c || (mem != SIF_HOST && mem != SIF_DEVICE)) return SIF_EINVAL;
  if (!c->inited) {
    set_err(c, "state not initialised");
    return SIF_ESTATE;
  }
  cudaSetDevice(c->cfg.device);
  size_t n = (size_t)ncell(c);
  int rc = SIF_OK;
  for (int m = 0; m < 4 && !rc; m++) {
    if (qN) rc = get_plane(c, qN + m * n, c->q[0][m], mem);
    if (qP && !rc) rc = get_plane(c, qP + m * n, c->q[1][m], mem);
  }
  if (phi && !rc) rc = get_plane(c, phi, c->phi, mem);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  return SIF_OK;
}

extern "C" int sif_set_state(sif_ctx *c, const double *qN, const double *qP, const double *phi,
                             double t, int mem) {
  if (!c || !qN || !qP || !phi || (mem != SIF_HOST && mem != SIF_DEVICE)) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  size_t n = (size_t)ncell(c);
  int rc = put_plane(c, c->phi, phi, mem);
  for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, c->q[0][m], qN + m * n, mem);
  for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, c->q[1][m], qP + m * n, mem);
  if (rc) return rc;
  geometry(c);
  c->hbuf[0] = t;
  CK(cudaMemcpyAsync(&c->sc->t, c->hbuf, sizeof(double), cudaMemcpyHostToDevice, c->st));
  rc = check_launch(c, "set_state");
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  c->inited = 1;
  return SIF_OK;
}

extern "C" int sif_integrals(sif_ctx *c, double *out) {
  if (!c || !out) return SIF_EINVAL;
  if (!c->inited) {
    set_err(c, "state not initialised");
    return SIF_ESTATE;
  }
  cudaSetDevice(c->cfg.device);
  launch_integrals(c->g, c->q[0], c->q[1], c->partial, 0, c->integ, c->st);
  int rc = check_launch(c, "integrals");
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->hbuf, c->integ, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  memcpy(out, c->hbuf, sizeof(double) * 8);
  return SIF_OK;
}

extern "C" int sif_get_time(sif_ctx *c, double *t) {
  if (!c || !t) return SIF_EINVAL;
  int rc = read_scalars(c);
  if (rc) return rc;
  *t = c->hsc->t;
  return SIF_OK;
}

// ---------------------------------------------------------------------
// checkpoint: header + 17 interior planes (qN, qP, wN, wP, phi)

struct CkptHeader {
  char magic[8];
  int version, nx, ny, nplanes;
  double t;
};

static const int kCkptPlanes = 17;

static double *ckpt_plane(sif_ctx *c, int i) {
  if (i < 4) return c->q[0][i];
  if (i < 8) return c->q[1][i - 4];
  if (i < 12) return c->w[0][i - 8];
  if (i < 16) return c->w[1][i - 12];
  return c->phi;
}

extern "C" int sif_save(sif_ctx *c, void *buf, size_t *len) {
  if (!c || !len) return SIF_EINVAL;
  size_t n = (size_t)ncell(c);
  size_t need = sizeof(CkptHeader) + sizeof(double) * n * kCkptPlanes;
  if (!buf) {
    *len = need;
    return SIF_OK;
  }
  if (*len < need) {
    set_err(c, "checkpoint buffer too small (%zu < %zu)", *len, need);
    return SIF_EINVAL;
  }
  if (!c->inited) {
    set_err(c, "state not initialised");
    return SIF_ESTATE;
  }
  cudaSetDevice(c->cfg.device);
  int rc = read_scalars(c);
  if (rc) return rc;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "SIFCKPT", 8);
  h.version = 1;
  h.nx = c->g.nx;
  h.ny = c->g.ny;
  h.nplanes = kCkptPlanes;
  h.t = c->hsc->t;
  memcpy(buf, &h, sizeof(h));
  double *out = (double *)((char *)buf + sizeof(h));
  for (int i = 0; i < kCkptPlanes && !rc; i++) rc = get_plane(c, out + i * n, ckpt_plane(c, i), SIF_HOST);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  *len = need;
  return SIF_OK;
}

extern "C" int sif_load(sif_ctx *c, const void *buf, size_t len) {
  if (!c || !buf) return SIF_EINVAL;
  size_t n = (size_t)ncell(c);
  size_t need = sizeof(CkptHeader) + sizeof(double) * n * kCkptPlanes;
  CkptHeader h;
  if (len < sizeof(h)) return SIF_EINVAL;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, "SIFCKPT", 8) != 0 || h.version != 1 || h.nx != c->g.nx ||
      h.ny != c->g.ny || h.nplanes != kCkptPlanes || len < need) {
    set_err(c, "checkpoint does not match this context");
    return SIF_EINVAL;
  }
  cudaSetDevice(c->cfg.device);
  const double *in = (const double *)((const char *)buf + sizeof(h));
  int rc = SIF_OK;
  for (int i = 0; i < kCkptPlanes && !rc; i++) rc = put_plane(c, ckpt_plane(c, i), in + i * n, SIF_HOST);
  if (rc) return rc;
  CK(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), c->st));
  c->hbuf[0] = h.t;
  CK(cudaMemcpyAsync(&c->sc->t, c->hbuf, sizeof(double), cudaMemcpyHostToDevice, c->st));
  geometry(c);
  rc = check_launch(c, "load");
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  c->inited = 1;
  return SIF_OK;
}

// ---------------------------------------------------------------------
// adjoint of the single-time-step method with its schedule frozen
//
// While a tape is active every single-dt step records what its frozen
// replay needs: the state, the stencil states it starts from (the
// extension's starting values), phi at its start, after stage 1 and at its
// end, dt and the Lax-Friedrichs speeds of both stages, and the stencil
// states both stages used.  The replay runs the same kernels with that
// schedule imposed; the adjoint takes the stages' stencil states from the
// tape, refreshes each stage's geometry from its level set and applies the
// transposed kernels in reverse order.

static double *tape_plane(sif_ctx *c, int step, int i) {
  return c->tape_planes + ((size_t)step * kTapePlanes + i) * c->NP;
}
static double *tape_scal(sif_ctx *c, int step) { return c->tape_scal + (size_t)step * 16; }
static unsigned char *tape_flags(sif_ctx *c, int step, int stage, int k) {
  return (unsigned char *)tape_plane(c, step, kTapeFlags) + (size_t)(stage * 2 + k) * c->NP;
}

static void d2d(sif_ctx *c, void *dst, const void *src, size_t bytes) {
  cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->st);
}

static void taped_step(sif_ctx *c) {
  const int s = c->tape_len;
  const size_t pb = sizeof(double) * c->NP;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      d2d(c, tape_plane(c, s, k * 4 + m), c->q[k][m], pb);
      d2d(c, tape_plane(c, s, 8 + k * 4 + m), c->w[k][m], pb);
    }
  d2d(c, tape_plane(c, s, 16), c->phi, pb);
  eval(c, c->q);
  launch_sched(SCHED_SINGLE_DT, c->sc, c->g.cfl, 0, 0, c->st);
  d2d(c, tape_scal(c, s), &c->sc->dt, sizeof(double));
  d2d(c, tape_scal(c, s) + 1, c->sc->lf, sizeof(c->sc->lf));
  for (int k = 0; k < 2; k++) d2d(c, tape_flags(c, s, 0, k), c->nostate[k], c->NP);
  TapeHook hook;
  hook.phi1 = tape_plane(c, s, 17);
  hook.lf2 = tape_scal(c, s) + 5;
  for (int k = 0; k < 2; k++) hook.flags2[k] = tape_flags(c, s, 1, k);
  for (int st = 0; st < 2; st++)
    for (int k = 0; k < 2; k++)
      for (int m = 0; m < 4; m++)
        hook.W[st][k][m] = tape_plane(c, s, (st == 0 ? kTapeW1 : kTapeW2) + k * 4 + m);
  single_step_after_eval(c, &c->sc->dt, &hook);
  d2d(c, tape_plane(c, s, 18), c->phi, pb);
  launch_sched(SCHED_T_SINGLE, c->sc, 0, 0, 0, c->st);
  c->tape_len++;
}

static int ensure_adj_scratch(sif_ctx *c) {
  if (c->adj_pool) return SIF_OK;
  const int nplanes = 24 + 8 + 8 + 40 + 8 + 17;
  size_t pb = sizeof(double) * c->NP;
  size_t bytes = pb * nplanes + sizeof(Scalars) + 256;
  if (cudaMalloc(&c->adj_pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->adj_pool = nullptr;
    set_err(c, "cannot allocate %zu bytes of adjoint scratch", bytes);
    return SIF_ECUDA;
  }
  double *p = (double *)c->adj_pool;
  auto take = [&]() {
    double *r = p;
    p += c->NP;
    return r;
  };
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      c->lamA[k][m] = take();
      c->lamB[k][m] = take();
      c->lamC[k][m] = take();
      c->lw[k][m] = take();
      c->prim[k][m] = take();
      c->sv_q[k][m] = take();
      c->sv_w[k][m] = take();
    }
  for (int q = 0; q < 40; q++) c->G[q] = take();
  for (int q = 0; q < 8; q++) c->SP[q] = take();
  c->sv_phi = take();
  c->sv_sc = (Scalars *)p;
  CK(cudaMemsetAsync(c->adj_pool, 0, bytes, c->st));
  return SIF_OK;
}

// the caller's state (q, stencil states, phi, scalars) around an adjoint call
static void save_state(sif_ctx *c) {
  const size_t pb = sizeof(double) * c->NP;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      d2d(c, c->sv_q[k][m], c->q[k][m], pb);
      d2d(c, c->sv_w[k][m], c->w[k][m], pb);
    }
  d2d(c, c->sv_phi, c->phi, pb);
  d2d(c, c->sv_sc, c->sc, sizeof(Scalars));
}

static void restore_state(sif_ctx *c) {
  const size_t pb = sizeof(double) * c->NP;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      d2d(c, c->q[k][m], c->sv_q[k][m], pb);
      d2d(c, c->w[k][m], c->sv_w[k][m], pb);
    }
  d2d(c, c->phi, c->sv_phi, pb);
  geometry(c);
  // the saved scalars hold the same list counts as the geometry just made
  d2d(c, c->sc, c->sv_sc, sizeof(Scalars));
}

static void set_phi(sif_ctx *c, const double *src) {
  d2d(c, c->phi, src, sizeof(double) * c->NP);
  geometry(c);
}

// recorded step `step` from the current q with its schedule imposed
static void frozen_forward(sif_ctx *c, int step) {
  const size_t pb = sizeof(double) * c->NP;
  double *sc = tape_scal(c, step);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) d2d(c, c->w[k][m], tape_plane(c, step, 8 + k * 4 + m), pb);
  set_phi(c, tape_plane(c, step, 16));
  d2d(c, &c->sc->dt, sc, sizeof(double));
  for (int k = 0; k < 2; k++) copy_planes(c, c->q0[k], c->q[k], 4);
  for (int s = 1; s <= 2; s++) {
    eval(c, c->q);
    d2d(c, c->sc->lf, sc + (s == 1 ? 1 : 5), sizeof(c->sc->lf));
    for (int k = 0; k < 2; k++) fv(c, k, s, c->q[k], c->q0[k], c->q[k], &c->sc->dt);
    set_phi(c, tape_plane(c, step, s == 1 ? 17 : 18));
    mix_both(c);
  }
}

// transposed right-hand side of the stage with stencil states W and LF
// speeds lf, applied to mu scaled by fac * dt, then primitive^T combined:
// out = ca A + cb B + J^T (fac dt mu).  The stage's geometry is in place.
static void adj_stage(sif_ctx *c, double *const W[2][4], const unsigned char *const flags[2],
                      const double *lf, const double *dtp, double fac, double *const mu[2][4],
                      double *const out[2][4], double *const A[2][4], double ca,
                      double *const B[2][4], double cb) {
  launch_ext_setup(c->g, c->alpha, c->phi, c->sx, c->sy, c->band_ev, &c->sc->n_band, c->bandmap,
                   c->ext_plan, ncell(c), band_work(c), flags, c->st);
  launch_adj_rhs(c->g, W, (const unsigned long long *)lf, dtp, fac, mu, c->ax, c->ay, c->phi,
                 c->sx, c->sy, c->cut, &c->sc->n_cut, ncell(c), c->G, c->SP, c->lw, c->st);
  launch_adj_extension(c->g, c->lw, c->ext_plan, ncell(c), band_work(c), c->band_ev,
                       &c->sc->n_band, c->bandmap, c->tmp, c->st);
  launch_adj_prim(c->g, W, c->alpha, flags, c->lw, out, A, ca, B, cb, c->st);
  dbg(c, "adjoint stage");
}

static void adj_mix(sif_ctx *c, double *const lam[2][4]) {
  launch_mix_adjoint(c->g, lam[0], lam[1], c->alpha, c->phi, c->band_ev, c->bandmap,
                     &c->sc->n_band, c->mix_plan, ncell(c), band_work(c), c->tmp, c->st);
}

// lamA = adjoint after step `step` -> lamC = adjoint before it; both
// stages' stencil states come from the tape
static void adjoint_step_impl(sif_ctx *c, int step) {
  double *sc = tape_scal(c, step);
  double *W1[2][4], *W2[2][4];
  const unsigned char *F1[2], *F2[2];
  for (int k = 0; k < 2; k++) {
    for (int m = 0; m < 4; m++) {
      W1[k][m] = tape_plane(c, step, kTapeW1 + k * 4 + m);
      W2[k][m] = tape_plane(c, step, kTapeW2 + k * 4 + m);
    }
    F1[k] = tape_flags(c, step, 0, k);
    F2[k] = tape_flags(c, step, 1, k);
  }
  // Q^{n+1} = mix(Q**) with the geometry of phi^{n+1}
  set_phi(c, tape_plane(c, step, 18));
  adj_mix(c, c->lamA);
  // Q** = Q^n / 2 + (Q1 + dt L(Q1)) / 2, stage-2 geometry
  set_phi(c, tape_plane(c, step, 17));
  adj_stage(c, W2, F2, sc + 5, sc, 0.5, c->lamA, c->lamB, c->lamA, 0.5, nullptr, 0.0);
  // Q1 = mix(Q*) with the same geometry
  adj_mix(c, c->lamB);
  // Q* = Q^n + dt L(Q^n), stage-1 geometry
  set_phi(c, tape_plane(c, step, 16));
  adj_stage(c, W1, F1, sc + 1, sc, 1.0, c->lamB, c->lamC, c->lamA, 0.5, c->lamB, 1.0);
}

static int put_state8(sif_ctx *c, double *const dst[2][4], const double *src, int mem) {
  size_t n = (size_t)ncell(c);
  int rc = SIF_OK;
  for (int k = 0; k < 2 && !rc; k++)
    for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, dst[k][m], src + (k * 4 + m) * n, mem);
  return rc;
}

static int get_state8(sif_ctx *c, double *dst, double *const src[2][4], int mem) {
  size_t n = (size_t)ncell(c);
  int rc = SIF_OK;
  for (int k = 0; k < 2 && !rc; k++)
    for (int m = 0; m < 4 && !rc; m++) rc = get_plane(c, dst + (k * 4 + m) * n, src[k][m], mem);
  return rc;
}

extern "C" int sif_tape_reset(sif_ctx *c, int capacity) {
  if (!c || capacity < 0) return SIF_EINVAL;
  if (c->cfg.rk_order != 2) {
    set_err(c, "the adjoint is defined for rk_order 2");
    return SIF_EINVAL;
  }
  if (c->cfg.weno_char || c->cfg.flux || c->cfg.sigma != 0.0 || c->cfg.mu[0] != 0.0 ||
      c->cfg.mu[1] != 0.0 || c->cfg.tait[0] || c->cfg.tait[1]) {
    set_err(c, "the adjoint is defined for the component-wise WENO-LF flux (weno_char 0, "
               "flux 0) of the inviscid stiffened-gas model without surface tension (sigma 0, "
               "mu 0, tait 0)");
    return SIF_EINVAL;
  }
  cudaSetDevice(c->cfg.device);
  CK(cudaStreamSynchronize(c->st));
  c->tape_len = 0;
  if (capacity == 0) {
    if (c->tape_planes) cudaFree(c->tape_planes);
    if (c->adj_pool) cudaFree(c->adj_pool);
    c->tape_planes = c->tape_scal = nullptr;
    c->adj_pool = nullptr;
    c->tape_cap = c->tape_alloc = 0;
    return SIF_OK;
  }
  if (capacity > c->tape_alloc) {
    if (c->tape_planes) cudaFree(c->tape_planes);
    c->tape_planes = c->tape_scal = nullptr;
    c->tape_alloc = 0;
    size_t bytes = sizeof(double) * ((size_t)capacity * kTapePlanes * c->NP + (size_t)capacity * 16);
    if (cudaMalloc(&c->tape_planes, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->tape_planes = nullptr;
      c->tape_cap = 0;
      set_err(c, "cannot allocate %zu bytes for a %d-step adjoint tape", bytes, capacity);
      return SIF_ECUDA;
    }
    c->tape_scal = c->tape_planes + (size_t)capacity * kTapePlanes * c->NP;
    c->tape_alloc = capacity;
  }
  c->tape_cap = capacity;
  return ensure_adj_scratch(c);
}

extern "C" int sif_tape_length(const sif_ctx *c, int *len) {
  if (!c || !len) return SIF_EINVAL;
  *len = c->tape_len;
  return SIF_OK;
}

static int adj_check(sif_ctx *c, int step, const void *a, const void *b, int mem) {
  if (!a || !b || (mem != SIF_HOST && mem != SIF_DEVICE)) return SIF_EINVAL;
  if (step < 0 || step >= c->tape_len) {
    set_err(c, "step %d not on the tape (%d recorded)", step, c->tape_len);
    return SIF_EINVAL;
  }
  if (!c->inited) {
    set_err(c, "state not initialised");
    return SIF_ESTATE;
  }
  return SIF_OK;
}

extern "C" int sif_replay_step(sif_ctx *c, int step, const double *q_in, double *q_out, int mem) {
  if (!c) return SIF_EINVAL;
  int rc = adj_check(c, step, q_in, q_out, mem);
  if (rc) return rc;
  cudaSetDevice(c->cfg.device);
  save_state(c);
  rc = put_state8(c, c->q, q_in, mem);
  if (rc) return rc;
  frozen_forward(c, step);
  rc = get_state8(c, q_out, c->q, mem);
  if (rc) return rc;
  CK(cudaMemcpyAsync(&c->hsc->err, &c->sc->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  restore_state(c);
  rc = check_launch(c, "replay");
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  if (c->hsc->err & DERR_NONPHYS) {
    set_err(c, "non-physical state (rho <= 0 or p + p_inf <= 0) in a real cell");
    return SIF_ENONPHYS;
  }
  return SIF_OK;
}

extern "C" int sif_adjoint_step(sif_ctx *c, int step, const double *lam_in, double *lam_out,
                                int mem) {
  if (!c) return SIF_EINVAL;
  int rc = adj_check(c, step, lam_in, lam_out, mem);
  if (rc) return rc;
  cudaSetDevice(c->cfg.device);
  save_state(c);
  rc = put_state8(c, c->lamA, lam_in, mem);
  if (rc) return rc;
  adjoint_step_impl(c, step);
  rc = get_state8(c, lam_out, c->lamC, mem);
  if (rc) return rc;
  restore_state(c);
  rc = check_launch(c, "adjoint step");
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  return SIF_OK;
}

extern "C" int sif_adjoint_init(sif_ctx *c, const double *phi, const double *pN, const double *pP,
                                const double *lam_q, double *lam_prim, int mem) {
  if (!c || !phi || !pN || !pP || !lam_q || !lam_prim || (mem != SIF_HOST && mem != SIF_DEVICE))
    return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  int rc = ensure_adj_scratch(c);
  if (rc) return rc;
  const bool had_state = c->inited;
  if (had_state) save_state(c);
  size_t n = (size_t)ncell(c);
  rc = put_plane(c, c->phi, phi, mem);
  for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, c->prim[0][m], pN + m * n, mem);
  for (int m = 0; m < 4 && !rc; m++) rc = put_plane(c, c->prim[1][m], pP + m * n, mem);
  if (!rc) rc = put_state8(c, c->lamA, lam_q, mem);
  if (rc) return rc;
  geometry(c);
  adj_mix(c, c->lamA);
  launch_adj_init(c->g, c->prim, c->alpha, c->lamA, c->lamC, c->st);
  rc = get_state8(c, lam_prim, c->lamC, mem);
  if (rc) return rc;
  if (had_state) restore_state(c);
  rc = check_launch(c, "adjoint init");
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->st));
  return SIF_OK;
}

// ---------------------------------------------------------------------
// measurement counters

extern "C" int sif_profile_enable(sif_ctx *c, int enable) {
  if (!c) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  int rc = read_scalars(c);
  if (rc) return rc;
  if (enable) {
    // re-arm the finite-volume launch timer and zero its sums
    struct {
      int timing;
      unsigned int done;
      unsigned long long t0, t1, ns, n;
    } z = {1, 0u, ~0ull, 0ull, 0ull, 0ull};
    static_assert(sizeof(z) == offsetof(Scalars, fv_launches) + sizeof(unsigned long long) -
                                   offsetof(Scalars, timing), "timer block layout");
    CK(cudaMemcpy((char *)c->sc + offsetof(Scalars, timing), &z, sizeof(z), cudaMemcpyHostToDevice));
    c->launches0 = device_launches();
    c->updates0 = c->hsc->updates;
    c->open0 = c->hsc->open_updates;
  } else {
    int zero = 0;
    CK(cudaMemcpy(&c->sc->timing, &zero, sizeof(int), cudaMemcpyHostToDevice));
  }
  c->profiling = enable ? 1 : 0;
  return SIF_OK;
}

extern "C" int sif_profile_read(sif_ctx *c, sif_profile *out) {
  if (!c || !out) return SIF_EINVAL;
  cudaSetDevice(c->cfg.device);
  int rc = read_scalars(c);
  if (rc) return rc;
  out->kernel_launches = (long long)(device_launches() - c->launches0);
  out->fv_launches = (long long)c->hsc->fv_launches;
  out->fv_ms = (double)c->hsc->fv_ns * 1e-6;
  out->fv_cell_updates = (long long)(c->hsc->updates - c->updates0);
  out->fv_open_updates = (long long)(c->hsc->open_updates - c->open0);
  return SIF_OK;
}

// ---------------------------------------------------------------------
// tile shape of the finite-volume kernel (chosen by the autotuner)

extern "C" int sif_set_tile_shape(sif_ctx *c, int tx, int ty) {
  if (!c) return SIF_EINVAL;
  if (!fv_shape_supported(tx, ty)) {
    set_err(c, "unsupported tile shape %d x %d", tx, ty);
    return SIF_EINVAL;
  }
  if (c->g.tx == tx && c->g.ty == ty) return SIF_OK;
  cudaSetDevice(c->cfg.device);
  CK(cudaStreamSynchronize(c->st));
  c->g.tx = tx;
  c->g.ty = ty;
  c->g.ntx = (c->g.nx + tx - 1) / tx;
  c->g.nty = (c->g.ny + ty - 1) / ty;
  free_graphs(c);
  if (c->inited) {
    geometry(c);  // tile lists for the new shape
    int rc = check_launch(c, "tile shape");
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->st));
  }
  return SIF_OK;
}

extern "C" int sif_get_tile_shape(const sif_ctx *c, int *tx, int *ty) {
  if (!c || !tx || !ty) return SIF_EINVAL;
  *tx = c->g.tx;
  *ty = c->g.ty;
  return SIF_OK;
}

// ---------------------------------------------------------------------
// limits of the bounded loops (both are baked into the captured graphs)

extern "C" int sif_set_limits(sif_ctx *c, int max_substeps, int newton_iters) {
  if (!c) return SIF_EINVAL;
  if (max_substeps > 1000000 || newton_iters > 10000) {
    set_err(c, "limits too large (%d sub-steps, %d Newton iterations)", max_substeps,
            newton_iters);
    return SIF_EINVAL;
  }
  cudaSetDevice(c->cfg.device);
  CK(cudaStreamSynchronize(c->st));
  if (max_substeps > 0) c->max_substeps = max_substeps;
  if (newton_iters > 0) c->g.newton_max = newton_iters;
  free_graphs(c);
  return SIF_OK;
}

// ---------------------------------------------------------------------
// batches of independent instances

struct sif_batch {
  int n;
  sif_ctx **ctx;
  cudaStream_t st;
  cudaGraphExec_t exec;
  std::vector<int> gens;  // instance graph generations the batch graph embeds
  std::vector<cudaEvent_t> events;  // fork/join of the batch capture
  int parent_ok;          // 0 after a failed attempt: launch instance graphs directly
  char err[256];
};

extern "C" int sif_batch_create(int n, const sif_config *cfgs, sif_batch **out) {
  if (!out) return SIF_EINVAL;
  *out = nullptr;
  if (n < 1 || !cfgs) return SIF_EINVAL;
  sif_batch *b = new (std::nothrow) sif_batch();
  if (!b) return SIF_ECUDA;
  b->n = n;
  b->parent_ok = 1;
  b->ctx = new (std::nothrow) sif_ctx *[n]();
  if (!b->ctx) {
    delete b;
    return SIF_ECUDA;
  }
  int rc = SIF_OK;
  for (int i = 0; i < n && rc == SIF_OK; i++) {
    sif_config f = cfgs[i];
    f.cuda_stream = nullptr;  // every instance gets its own stream
    rc = sif_create(&f, &b->ctx[i]);
    // the instances' kernels run side by side: the extension sweeps go one
    // launch per sweep or two (small blocks that share SMs) rather than as
    // band tiles whose CTAs each take a whole SM's registers (measured on
    // the 256-instance batch: 244 against 274 ms a cycle)
    if (rc == SIF_OK) b->ctx[i]->ext_blocked = 0;
  }
  if (rc == SIF_OK && cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
    rc = SIF_ECUDA;
  if (rc != SIF_OK) {
    sif_batch_destroy(b);
    return rc;
  }
  snprintf(b->err, sizeof(b->err), "ok");
  *out = b;
  return SIF_OK;
}

extern "C" int sif_batch_instance(sif_batch *b, int i, sif_ctx **out) {
  if (!b || !out || i < 0 || i >= b->n) return SIF_EINVAL;
  *out = b->ctx[i];
  return SIF_OK;
}

extern "C" const char *sif_batch_last_error(const sif_batch *b) { return b ? b->err : "null batch"; }

extern "C" void sif_batch_destroy(sif_batch *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto ev : b->events) cudaEventDestroy(ev);
  if (b->ctx)
    for (int i = 0; i < b->n; i++) sif_destroy(b->ctx[i]);
  delete[] b->ctx;
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

// one graph whose parallel branches are the instances' cycles: a single
// capture on the batch stream forks every instance stream off it, captures
// that instance's cycle (with its conditional nodes) on it, and joins back
static int batch_build(sif_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  if (b->events.empty()) {
    b->events.resize(b->n + 1);
    for (auto &ev : b->events) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->events[b->n], b->st);
  for (int i = 0; i < b->n && e == cudaSuccess; i++) {
    sif_ctx *c = b->ctx[i];
    e = cudaStreamWaitEvent(c->st, b->events[b->n], 0);
    if (e != cudaSuccess) break;
    int saved = c->band_work;
    c->band_work = c->graph_bucket;
    c->gerr = 0;
    c->capturing = 1;
    c->cap_depth = 0;
    capture_cycle(c);
    c->capturing = 0;
    c->band_work = saved;
    if (c->gerr) e = (cudaError_t)c->gerr;
    if (e == cudaSuccess) e = cudaEventRecord(b->events[i], c->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->events[i], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->exec = nullptr;
    b->parent_ok = 0;
    return SIF_ECUDA;
  }
  b->gens.resize(b->n);
  for (int i = 0; i < b->n; i++) b->gens[i] = b->ctx[i]->graph_gen;
  return SIF_OK;
}

extern "C" int sif_batch_step_multi_dt(sif_batch *b, int ncycles, long long *cell_updates,
                                       long long *open_updates) {
  if (!b || ncycles < 0) return SIF_EINVAL;
  std::vector<Upd> upd0(b->n);
  bool rebuild = !b->exec;
  for (int i = 0; i < b->n; i++) {
    sif_ctx *c = b->ctx[i];
    if (!c->inited) {
      snprintf(b->err, sizeof(b->err), "instance %d: not initialised", i);
      return SIF_ESTATE;
    }
    int rc = begin_call(c, 0.0, &upd0[i]);
    if (rc == SIF_OK) rc = ensure_graphs(c);
    if (rc != SIF_OK) {
      snprintf(b->err, sizeof(b->err), "instance %d: graph set-up failed: %.200s", i, c->err);
      return rc == SIF_OK ? SIF_ECUDA : rc;
    }
    if (b->exec && b->gens.size() == (size_t)b->n && b->gens[i] != c->graph_gen) rebuild = true;
  }
  if (rebuild && b->parent_ok) batch_build(b);
  for (int i = 0; i < b->n; i++) cudaStreamSynchronize(b->ctx[i]->st);
  for (int n = 0; n < ncycles; n++) {
    if (b->exec) {
      if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) break;
    } else {
      for (int i = 0; i < b->n; i++) cudaGraphLaunch(b->ctx[i]->g_cycle, b->ctx[i]->st);
    }
  }
  cudaError_t e = b->exec ? cudaStreamSynchronize(b->st) : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    snprintf(b->err, sizeof(b->err), "batch cycle: %s", cudaGetErrorString(e));
    return SIF_ECUDA;
  }
  long long total = 0, total_open = 0;
  int first_rc = SIF_OK;
  for (int i = 0; i < b->n; i++) {
    int rc = finish(b->ctx[i], nullptr, upd0[i]);
    total += (long long)(b->ctx[i]->hsc->updates - upd0[i].tile);
    total_open += (long long)(b->ctx[i]->hsc->open_updates - upd0[i].open);
    if (rc != SIF_OK && first_rc == SIF_OK) {
      first_rc = rc;
      snprintf(b->err, sizeof(b->err), "instance %d: %.200s", i, b->ctx[i]->err);
    }
  }
  if (cell_updates) *cell_updates = total;
  if (open_updates) *open_updates = total_open;
  return first_rc;
}

extern "C" int sif_batch_one_graph(const sif_batch *b) { return b && b->exec ? 1 : 0; }
