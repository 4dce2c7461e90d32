// kernels_plan.cu -- narrow-band work of the interaction step with the
// per-cell decisions taken once: the interaction band with a cell -> band
// position map, the upwind neighbours and weights of the extension
// (Sec. 2.3: stencil states of both fluids and the level-set velocity),
// and the small-cell mixing sources with their targets and weights
// (Sec. 2.2).  The Jacobi sweeps and the mixing gather then only read the
// plans, both fluids per launch.
//
// Compiled without FMA contraction, like the other branch-taking kernels.
#include "sif_internal.cuh"

static int blocks_for(int n, int per) {
  int b = (n + per - 1) / per;
  if (b > 2432) b = 2432;
  return b < 1 ? 1 : b;
}

// ---------------------------------------------------------------------
// interaction band and its map

int ext_tiles(const Grid &g) {
  return ((g.nx + SIF_ETILE - 1) / SIF_ETILE) * ((g.ny + SIF_ETILE - 1) / SIF_ETILE);
}

// Blocks [0, ext_tiles): one SIF_ETILE x SIF_ETILE tile each, whose band
// cells join the band list (warp-aggregated positions) and the map, and
// which joins the extension tile list if it holds any.  Blocks from
// ext_tiles on: one finite-volume tile each, which joins fluid k's tile
// list if a cell of the tile or of its one-cell ring (ghosts included) lies
// on fluid k's side (where fluid k can hold an open face).  Both read only
// phi.
__global__ void k_band_tiles(Grid g, const double *__restrict__ p, int *band, int *map,
                             int *etiles, int *t0, int *t1, Scalars *sc) {
  SIF_TICK();
  const int tilesx = (g.nx + SIF_ETILE - 1) / SIF_ETILE;
  const int nt = tilesx * ((g.ny + SIF_ETILE - 1) / SIF_ETILE);
  if ((int)blockIdx.x < nt) {
    const int i = (blockIdx.x % tilesx) * SIF_ETILE + (threadIdx.x % SIF_ETILE);
    const int j = (blockIdx.x / tilesx) * SIF_ETILE + (threadIdx.x / SIF_ETILE);
    bool in = false;
    int c = 0;
    if (i < g.nx && j < g.ny) {
      c = gidx(g, i, j);
      in = fabs(p[c]) < g.band * g.h;
    }
    unsigned mask = __ballot_sync(0xffffffffu, in);
    if (mask) {
      int lane = threadIdx.x & 31, lead = __ffs(mask) - 1;
      int base = 0;
      if (lane == lead) base = atomicAdd(&sc->n_band, __popc(mask));
      base = __shfl_sync(0xffffffffu, base, lead);
      if (in) {
        int pos = base + __popc(mask & ((1u << lane) - 1u));
        band[pos] = c;
        map[c] = pos;
      }
    }
    if (__syncthreads_or(in) && threadIdx.x == 0)
      etiles[atomicAdd(&sc->n_etile, 1)] = blockIdx.x;
    return;
  }
  const int tile = blockIdx.x - nt;
  const int tx = tile % g.ntx, ty = tile / g.ntx;
  const int i0 = tx * g.tx - 1, j0 = g.dim == 2 ? ty * g.ty - 1 : 0;
  const int wy = g.dim == 2 ? g.ty + 2 : 1;
  int any_pos = 0, any_neg = 0;
  for (int r = threadIdx.x; r < (g.tx + 2) * wy; r += blockDim.x) {
    int i = i0 + r % (g.tx + 2), j = j0 + r / (g.tx + 2);
    if (i < -1 || i > g.nx || j < -1 || j > g.ny) continue;
    double v = p[gidx(g, i, j)];
    if (v >= 0.0) any_pos = 1;
    else any_neg = 1;
  }
  any_pos = __syncthreads_or(any_pos);
  any_neg = __syncthreads_or(any_neg);
  if (threadIdx.x == 0) {
    if (any_neg) t0[atomicAdd(&sc->n_tiles[0], 1)] = tile;
    if (any_pos) t1[atomicAdd(&sc->n_tiles[1], 1)] = tile;
  }
}

// the whole map is cleared (not only the previous band's entries): a reset
// of the device scalars (initialisation, checkpoint restore) loses the
// previous band's count, and the clear must not depend on it
void launch_band_tiles(const Grid &g, const double *phi, int *band, int *map, int *etiles,
                       int *tiles0, int *tiles1, Scalars *sc, cudaStream_t st) {
  static_assert(offsetof(Scalars, n_tiles) == offsetof(Scalars, n_band) + 2 * sizeof(int),
                "the band, extension-tile and finite-volume tile counts are cleared together");
  cudaMemsetAsync(map, 0xff, sizeof(int) * (size_t)g.PX * g.PY, st);
  cudaMemsetAsync(&sc->n_band, 0, 4 * sizeof(int), st);
  launch_k(k_band_tiles, ext_tiles(g) + g.ntx * g.nty, SIF_ETILE * SIF_ETILE, 0, st, g, phi,
           band, map, etiles, tiles0, tiles1, sc);
  sif_note_launches(1);
}

// Jacobi sweeps of fields [f0, f0 + nf) (blockIdx.y selects the field),
// ping-ponging between two band-indexed buffers: sweep 0 reads the planes,
// later sweeps read the previous sweep's buffer for band neighbours and the
// planes for neighbours outside the band (whose values never change)
struct ExtFields {
  double *p[3][4];
  int ncomp[3];
  double gamma[2], pinf[2];
};

// the upwind-weighted mean of a target's neighbour values x (weight wx,
// present if hx) and y (wy, hy): one product and one fused multiply-add,
// the same operations in every form of the extension
__device__ __forceinline__ double ext_mean(bool hx, double wx, double x, bool hy, double wy,
                                           double y) {
  if (hx && hy) return __fma_rn(wy, y, wx * x);
  return hx ? wx * x : wy * y;
}

// ---------------------------------------------------------------------
// extension plans: for every band cell and each of the three extended
// fields (W_N, W_P, level-set velocity) the upwind x and y neighbours and
// their normalised weights, or "not a target"

__global__ void k_ext_setup(Grid g, const double *__restrict__ alpha,
                            const double *__restrict__ phi, const double *__restrict__ sx,
                            const double *__restrict__ sy, const int *__restrict__ band,
                            const int *nband, const int *__restrict__ map, ExtPlan *plan,
                            int cap, const unsigned char *__restrict__ ns0,
                            const unsigned char *__restrict__ ns1, ExtFields F, double *sweep0,
                            int copy) {
  SIF_TICK();
  const int f = blockIdx.y;  // field: W_N, W_P, level-set velocity
  int n = *nband;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    double nxv, nyv;
    unit_normal(g, phi, i, j, nxv, nyv);
    {
      ExtPlan pl = {-1, -1, -1, -1, 0.0, 0.0};
      bool target;
      double dx_, dy_;
      if (f < 2) {
        target = !(vol_k(alpha, f, c) > SIF_ALPHA_REAL) || (f == 0 ? ns0 : ns1)[c];
        // toward fluid f: its normal points into it
        dx_ = f == 0 ? -nxv : nxv;
        dy_ = f == 0 ? -nyv : nyv;
      } else {
        target = (sx[c] == 0.0 && sy[c] == 0.0);
        // toward the interface from either side
        dx_ = phi[c] >= 0.0 ? -nxv : nxv;
        dy_ = phi[c] >= 0.0 ? -nyv : nyv;
      }
      if (target) {
        int six = dx_ >= 0.0 ? 1 : -1, siy = dy_ >= 0.0 ? 1 : -1;
        double wx = fabs(dx_) / g.dx;
        double wy = g.dim == 2 ? fabs(dy_) / g.dy : 0.0;
        if (!inside(g, i + six, j)) wx = 0.0;
        if (!inside(g, i, j + siy)) wy = 0.0;
        double den = wx + wy;
        if (den > 0.0) {
          if (wx > 0.0) {
            pl.cx = gidx(g, i + six, j);
            pl.bx = map[pl.cx];
            pl.wx = wx / den;
          }
          if (wy > 0.0) {
            pl.cy = gidx(g, i, j + siy);
            pl.by = map[pl.cy];
            pl.wy = wy / den;
          }
        }
      }
      plan[(size_t)f * cap + idx] = pl;
      // the first sweep of the stencil states (k_ext_sweep without a
      // previous sweep), while the plan is at hand; for the blocked
      // extension the band cells' own values instead
      if (sweep0 && f < 2) {
#pragma unroll
        for (int m = 0; m < 4; m++) {
          const double *a = F.p[f][m];
          double v;
          if (copy || (pl.cx < 0 && pl.cy < 0)) {
            v = a[c];
          } else {
            v = ext_mean(pl.cx >= 0, pl.wx, pl.cx >= 0 ? a[pl.cx] : 0.0, pl.cy >= 0, pl.wy,
                         pl.cy >= 0 ? a[pl.cy] : 0.0);
          }
          sweep0[(size_t)f * 4 * cap + (size_t)m * cap + idx] = v;
        }
      }
    }
  }
}

void launch_ext_setup(const Grid &g, const double *alpha, const double *phi, const double *sx,
                      const double *sy, const int *band, const int *nband, const int *map,
                      ExtPlan *plan, int cap, int work, const unsigned char *const nostate[2],
                      cudaStream_t st, double *const wN[4], double *const wP[4],
                      double *sweep0, int copy) {
  ExtFields F = {};
  if (sweep0)
    for (int m = 0; m < 4; m++) {
      F.p[0][m] = wN[m];
      F.p[1][m] = wP[m];
    }
  // one block row per field
  launch_k(k_ext_setup, dim3(blocks_for(work, 64), 3), 64, 0, st, 
      g, alpha, phi, sx, sy, band, nband, map, plan, cap, nostate[0], nostate[1], F, sweep0,
      copy);
  sif_note_launches(1);
}


// fold a block's wave speeds of extended stencil states into the
// Lax-Friedrichs maxima of fluid f (every thread of the block calls it)
__device__ void ext_fold_lf(double lx, double ly, unsigned long long *lf) {
  __shared__ double sa[32], sb[32];
  lx = warp_max(lx);
  ly = warp_max(ly);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = lx;
    sb[wid] = ly;
  }
  __syncthreads();
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    lx = lane < nw ? sa[lane] : 0.0;
    ly = lane < nw ? sb[lane] : 0.0;
    lx = warp_max(lx);
    ly = warp_max(ly);
    if (lane == 0) {
      atomic_max_pos(&lf[0], lx);
      atomic_max_pos(&lf[1], ly);
    }
  }
}

// value of band cell `cell` (band position bp, plan px) after one Jacobi
// sweep from the values b of the previous sweep (the planes a when b is
// null): the upwind-weighted mean of its upwind neighbours for a target,
// its own value otherwise
__device__ __forceinline__ double ext_one(const ExtPlan &px, int bp, int cell, const double *a,
                                          const double *b) {
  if (px.cx < 0 && px.cy < 0) return b ? b[bp] : a[cell];
  const double x = px.cx >= 0 ? ((b && px.bx >= 0) ? b[px.bx] : a[px.cx]) : 0.0;
  const double y = px.cy >= 0 ? ((b && px.by >= 0) ? b[px.by] : a[px.cy]) : 0.0;
  return ext_mean(px.cx >= 0, px.wx, x, px.cy >= 0, px.wy, y);
}

// S (1 or 2) Jacobi sweeps in one launch.  With S = 2 a target recomputes
// its upwind neighbours' intermediate values from their plans (the same
// operations as the sweep in between), which takes one dependent load
// level more and one launch fewer.  With writeback (a launch whose first
// sweep is not the first: band cells then read only the previous sweep's
// buffer) the results go straight to the planes, and the extended stencil
// states fold their wave speeds into the Lax-Friedrichs maxima, as
// k_ext_scatter would.  The band position and plan of a thread's first
// cell are loaded together with the band count.
template <int S>
__global__ void k_ext_sweep(ExtFields F, int f0, const ExtPlan *__restrict__ plan, int cap,
                            const int *__restrict__ band, const int *nband,
                            const double *__restrict__ src, double *dst, int writeback,
                            const double *__restrict__ alpha,
                            const unsigned char *__restrict__ ns0,
                            const unsigned char *__restrict__ ns1, Scalars *sc) {
  SIF_TICK();
  const int f = f0 + blockIdx.y;
  const int nc = F.ncomp[f];
  const ExtPlan *P = plan + (size_t)f * cap;
  const size_t slot = (size_t)blockIdx.y * 4 * cap;
  const int idx0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool inb = idx0 < cap;
  const int c0 = inb ? band[idx0] : 0;
  const ExtPlan pl0 = inb ? P[idx0] : ExtPlan{-1, -1, -1, -1, 0.0, 0.0};
  const int n = *nband;
  const bool fold = writeback && f < 2;
  double lx = 0.0, ly = 0.0;
  for (int idx = idx0; idx < n; idx += gridDim.x * blockDim.x) {
    int c = idx == idx0 ? c0 : band[idx];
    ExtPlan pl = idx == idx0 ? pl0 : P[idx];
    // the upwind neighbours' plans (two sweeps: their intermediate values)
    const bool hx = S == 2 && pl.cx >= 0 && pl.bx >= 0;
    const bool hy = S == 2 && pl.cy >= 0 && pl.by >= 0;
    ExtPlan px = {-1, -1, -1, -1, 0.0, 0.0}, py = {-1, -1, -1, -1, 0.0, 0.0};
    if (hx) px = P[pl.bx];
    if (hy) py = P[pl.by];
    double out[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < 4; m++) {
      if (m >= nc) break;
      const double *a = F.p[f][m];
      const double *b = src ? src + slot + (size_t)m * cap : nullptr;
      double v;
      if (S == 1) {
        v = ext_one(pl, idx, c, a, b);
      } else if (pl.cx < 0 && pl.cy < 0) {
        v = b ? b[idx] : a[c];
      } else {
        const double x = pl.cx >= 0 ? (hx ? ext_one(px, pl.bx, pl.cx, a, b) : a[pl.cx]) : 0.0;
        const double y = pl.cy >= 0 ? (hy ? ext_one(py, pl.by, pl.cy, a, b) : a[pl.cy]) : 0.0;
        v = ext_mean(pl.cx >= 0, pl.wx, x, pl.cy >= 0, pl.wy, y);
      }
      out[m] = v;
    }
    if (writeback) {
#pragma unroll
      for (int m = 0; m < 4; m++)
        if (m < nc) F.p[f][m][c] = out[m];
      if (fold && (!(vol_k(alpha, f, c) > SIF_ALPHA_REAL) || (f == 0 ? ns0 : ns1)[c])) {
        double cs = sqrt(fmax(F.gamma[f] * (out[3] + F.pinf[f]) / out[0], 0.0));
        lx = fmax(lx, fabs(out[1]) + cs);
        ly = fmax(ly, fabs(out[2]) + cs);
      }
    } else {
#pragma unroll
      for (int m = 0; m < 4; m++)
        if (m < nc) dst[slot + (size_t)m * cap + idx] = out[m];
    }
  }
  if (fold) ext_fold_lf(lx, ly, sc->lf[f]);
}

// write the last sweep back; for the stencil states fold the extended
// cells' wave speeds into the Lax-Friedrichs maxima
__global__ void k_ext_scatter(Grid g, ExtFields F, int f0, int cap, const int *__restrict__ band,
                              const int *nband, const double *buf,
                              const double *__restrict__ alpha,
                              const unsigned char *__restrict__ ns0,
                              const unsigned char *__restrict__ ns1, Scalars *sc) {
  SIF_TICK();
  int n = *nband;
  int f = f0 + blockIdx.y;
  int nc = F.ncomp[f];
  const double *in = buf + (size_t)blockIdx.y * 4 * cap;
  double lx = 0.0, ly = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    for (int m = 0; m < nc; m++) F.p[f][m][c] = in[(size_t)m * cap + idx];
    if (f < 2 && (!(vol_k(alpha, f, c) > SIF_ALPHA_REAL) || (f == 0 ? ns0 : ns1)[c])) {
      double r = in[idx], u = in[(size_t)cap + idx], v = in[(size_t)2 * cap + idx],
             p = in[(size_t)3 * cap + idx];
      double cs = sqrt(fmax(g.gamma[f] * (p + g.pinf[f]) / r, 0.0));
      lx = fmax(lx, fabs(u) + cs);
      ly = fmax(ly, fabs(v) + cs);
    }
  }
  if (f < 2) ext_fold_lf(lx, ly, sc->lf[f]);
}

void launch_ext_sweeps(const Grid &g, double *const wN[4], double *const wP[4], double *ul0,
                       double *ul1, int f0, int nf, const ExtPlan *plan, int cap, int work,
                       const int *band, const int *nband, double *tmp, const double *alpha,
                       const unsigned char *const nostate[2], Scalars *sc, cudaStream_t st,
                       int first_done) {
  ExtFields F;
  for (int m = 0; m < 4; m++) {
    F.p[0][m] = wN[m];
    F.p[1][m] = wP[m];
    F.p[2][m] = m == 0 ? ul0 : (m == 1 ? ul1 : nullptr);
  }
  F.ncomp[0] = F.ncomp[1] = 4;
  F.ncomp[2] = 2;
  for (int k = 0; k < 2; k++) {
    F.gamma[k] = g.gamma[k];
    F.pinf[k] = g.pinf[k];
  }
  dim3 grid(blocks_for(work, 64), nf);
  double *buf[2] = {tmp, tmp + (size_t)8 * cap};
  // first_done: sweep 0 is already in buf[0] (written by k_ext_setup).
  // The stencil states' remaining sweeps (on the interaction step's
  // critical path) go two per launch, one first when their number is odd;
  // the level-set velocity's (a graph branch beside the finite-volume
  // stage, where a heavier kernel slows the stage) one per launch.  The
  // last launch writes the planes itself unless its first sweep is the
  // very first (which reads band neighbours from the planes it would
  // overwrite), in which case the scatter writes them back.
  const double *src = first_done ? buf[0] : nullptr;
  int cur = first_done ? 1 : 0;
  const int iters = g.ext_iters;
  int remaining = iters - (first_done ? 1 : 0);
  int launched = 0;
  while (remaining > 0) {
    const int S = (f0 == 0 && remaining % 2 == 0) ? 2 : 1;
    const int wb = remaining == S && src != nullptr;
    if (S == 1)
      launch_k(k_ext_sweep<1>, grid, 64, 0, st, F, f0, plan, cap, band, nband, src, buf[cur], wb,
                                          alpha, nostate[0], nostate[1], sc);
    else
      launch_k(k_ext_sweep<2>, grid, 64, 0, st, F, f0, plan, cap, band, nband, src, buf[cur], wb,
                                          alpha, nostate[0], nostate[1], sc);
    remaining -= S;
    launched++;
    if (wb) {
      src = nullptr;  // written back
      break;
    }
    src = buf[cur];
    cur ^= 1;
  }
  if (src) {
    launch_k(k_ext_scatter, grid, 64, 0, st, g, F, f0, cap, band, nband, src, alpha, nostate[0],
                                        nostate[1], sc);
    launched++;
  }
  sif_note_launches(launched);
}

// ---------------------------------------------------------------------
// blocked extension: all Jacobi sweeps of a band tile in shared memory.
// A CTA loads its tile with a halo of g.ext_iters cells (every field value
// there: band cells at their pre-extension values, others constant), the
// targets' upwind neighbours and weights, and runs the sweeps in place.  A
// target on the region's rim whose neighbour lies outside keeps a stale
// value; staleness moves one cell per sweep, so after g.ext_iters sweeps
// the tile itself holds the values the band-wide Jacobi iteration gives,
// each computed by the same operations in the same order.
//
// Where the pre-extension band values come from decides where the results
// may go.  The stencil states' band values are copied to a band-indexed
// buffer by the plan kernel (k_ext_setup): the CTAs read band cells only
// there and other cells only from the planes, so each writes its tile's
// band values straight into the planes (and folds their wave speeds).  The
// level-set velocity's band values are read from the planes, so its
// results go to a band-indexed buffer and a second launch writes them back.

constexpr int EXT_THREADS = 512;
constexpr int EXT_RW_MAX = SIF_ETILE + 2 * SIF_EXT_BLOCKED_MAX;
// region cells (and targets) a thread holds
constexpr int EXT_PER = (EXT_RW_MAX * EXT_RW_MAX + EXT_THREADS - 1) / EXT_THREADS;
// the largest distance of a region cell to the region's rim
constexpr int EXT_DMAX = (EXT_RW_MAX - 1) / 2;

static size_t ext_blocked_smem(int nc, int H) {
  const size_t rw = SIF_ETILE + 2 * H, r = rw * rw;
  // values, then per target: two weights, packed neighbours, region index;
  // per region cell its band position
  return r * (sizeof(double) * (nc + 2) + 3 * sizeof(int));
}

bool ext_blocked_ok(const Grid &g) {
  return g.ext_iters >= 1 && g.ext_iters <= SIF_EXT_BLOCKED_MAX;
}

// DIRECT: band values from bandin (4 x cap per field, band-indexed), results
// into the planes with the wave-speed fold; else band values from the
// planes, results into out (4 x cap per field)
template <int NC, bool DIRECT>
__global__ void __launch_bounds__(EXT_THREADS)
k_ext_blocked(Grid g, ExtFields F, int f0, const ExtPlan *__restrict__ plan, int cap,
              const int *__restrict__ etiles, const int *nband, const int *__restrict__ map,
              const double *__restrict__ bandin, double *out, const double *__restrict__ alpha,
              const unsigned char *__restrict__ ns0, const unsigned char *__restrict__ ns1,
              Scalars *sc) {
  SIF_TICK();
  extern __shared__ double esm[];
  __shared__ int s_hist[EXT_DMAX + 1], s_start[EXT_DMAX + 1];
  const int f = f0 + blockIdx.y;
  const int H = g.ext_iters, RW = SIF_ETILE + 2 * H, R = RW * RW;
  double *val = esm;              // NC x R
  double *wxs = val + NC * R;     // per target
  double *wys = wxs + R;
  int *nbs = (int *)(wys + R);    // neighbours' region indices + 1 (x low, y high half)
  int *tls = nbs + R;             // target's region index
  int *bps = tls + R;             // region cell's band position (-1: none)
  const ExtPlan *P = plan + (size_t)f * cap;
  const double *in = DIRECT ? bandin + (size_t)f * 4 * cap : nullptr;
  double *o = DIRECT ? nullptr : out + (size_t)blockIdx.y * 4 * cap;
  const unsigned char *ns = f == 0 ? ns0 : ns1;
  const int tilesx = (g.nx + SIF_ETILE - 1) / SIF_ETILE;
  const int nt_tiles = nband[1];
  const int tid = threadIdx.x;
  double lx = 0.0, ly = 0.0;
  for (int q = blockIdx.x; q < nt_tiles; q += gridDim.x) {
    const int et = etiles[q];
    const int ri0 = (et % tilesx) * SIF_ETILE - H, rj0 = (et / tilesx) * SIF_ETILE - H;
    for (int d = tid; d <= EXT_DMAX; d += EXT_THREADS) s_hist[d] = 0;
    // the region's band positions and plane values, then the band cells'
    // plans (and buffered values): two dependent load levels in all
    int cc[EXT_PER], bp[EXT_PER];
    double v[EXT_PER][NC];
#pragma unroll
    for (int l = 0; l < EXT_PER; l++) {
      const int r = tid + l * EXT_THREADS;
      const int i = ri0 + r % RW, j = rj0 + r / RW;
      const bool ok = r < R && i >= 0 && j >= 0 && i < g.nx && j < g.ny;
      cc[l] = ok ? gidx(g, i, j) : -1;
      bp[l] = ok ? map[cc[l]] : -1;
    }
    ExtPlan pl[EXT_PER];
#pragma unroll
    for (int l = 0; l < EXT_PER; l++) {
      pl[l] = ExtPlan{-1, -1, -1, -1, 0.0, 0.0};
      if (bp[l] >= 0) pl[l] = P[bp[l]];
      // band values (the planes' band cells are being written by other
      // CTAs in the direct form), else the planes
      const bool buffered = DIRECT && bp[l] >= 0;
#pragma unroll
      for (int m = 0; m < NC; m++)
        v[l][m] = buffered ? in[(size_t)m * cap + bp[l]] : (cc[l] >= 0 ? F.p[f][m][cc[l]] : 0.0);
    }
    __syncthreads();  // s_hist is clear
    // targets sorted by their distance to the region's rim, the farthest
    // first: sweep s (0-based) updates only those at distance s + 1 or more
    // (the others are stale by then whatever they hold), a prefix of the
    // list
    int dist[EXT_PER], nxs[EXT_PER], nys[EXT_PER];
#pragma unroll
    for (int l = 0; l < EXT_PER; l++) {
      const int r = tid + l * EXT_THREADS;
      dist[l] = -1;
      if (r >= R) continue;
      bps[r] = bp[l];
#pragma unroll
      for (int m = 0; m < NC; m++) val[m * R + r] = v[l][m];
      if (pl[l].cx < 0 && pl[l].cy < 0) continue;
      const int li = r % RW, lj = r / RW, c = cc[l];
      int nx_ = -1, ny_ = -1;
      bool rim = false;
      if (pl[l].cx >= 0) {
        const int d = pl[l].cx - c;  // +-1
        if (li + d < 0 || li + d >= RW) rim = true;
        else nx_ = r + d;
      }
      if (pl[l].cy >= 0) {
        const int d = (pl[l].cy - c) / g.PX;  // +-1
        if (lj + d < 0 || lj + d >= RW) rim = true;
        else ny_ = r + d * RW;
      }
      if (rim) continue;
      dist[l] = min(min(li, lj), min(RW - 1 - li, RW - 1 - lj));
      nxs[l] = nx_;
      nys[l] = ny_;
      atomicAdd(&s_hist[dist[l]], 1);
    }
    __syncthreads();
    if (tid == 0) {
      // s_start[d]: targets farther than d from the rim (they come first)
      int acc = 0;
      for (int d = EXT_DMAX; d >= 0; d--) {
        s_start[d] = acc;
        acc += s_hist[d];
      }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < EXT_PER; l++) {
      if (dist[l] < 0) continue;
      const int k = s_start[dist[l]] + atomicAdd(&s_hist[dist[l]], -1) - 1;
      tls[k] = tid + l * EXT_THREADS;
      wxs[k] = pl[l].wx;
      wys[k] = pl[l].wy;
      nbs[k] = (nxs[l] + 1) | ((nys[l] + 1) << 16);
    }
    __syncthreads();
    for (int s = 0; s < H; s++) {
      const int nt = s_start[s];
      double nv[EXT_PER][NC];
#pragma unroll
      for (int kk = 0; kk < EXT_PER; kk++) {
        const int k = tid + kk * EXT_THREADS;
        if (k < nt) {
          const int nb = nbs[k], nx_ = (nb & 0xffff) - 1, ny_ = (nb >> 16) - 1;
          const double wx = wxs[k], wy = wys[k];
#pragma unroll
          for (int m = 0; m < NC; m++)
            nv[kk][m] = ext_mean(nx_ >= 0, wx, nx_ >= 0 ? val[m * R + nx_] : 0.0, ny_ >= 0, wy,
                                 ny_ >= 0 ? val[m * R + ny_] : 0.0);
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < EXT_PER; kk++) {
        const int k = tid + kk * EXT_THREADS;
        if (k < nt) {
          const int r = tls[k];
#pragma unroll
          for (int m = 0; m < NC; m++) val[m * R + r] = nv[kk][m];
        }
      }
      __syncthreads();
    }
    // the tile's band cells
    for (int r = tid; r < SIF_ETILE * SIF_ETILE; r += EXT_THREADS) {
      const int li = H + r % SIF_ETILE, lj = H + r / SIF_ETILE;
      const int i = ri0 + li, j = rj0 + lj;
      if (i >= g.nx || j >= g.ny) continue;
      const int rr = lj * RW + li, b = bps[rr];
      if (b < 0) continue;
      if (DIRECT) {
        const int c = gidx(g, i, j);
#pragma unroll
        for (int m = 0; m < NC; m++) F.p[f][m][c] = val[m * R + rr];
        if (!(vol_k(alpha, f, c) > SIF_ALPHA_REAL) || ns[c]) {
          const double rho = val[rr], u = val[R + rr], vv = val[2 * R + rr],
                       p = val[3 * R + rr];
          const double cs = sqrt(fmax(F.gamma[f] * (p + F.pinf[f]) / rho, 0.0));
          lx = fmax(lx, fabs(u) + cs);
          ly = fmax(ly, fabs(vv) + cs);
        }
      } else {
#pragma unroll
        for (int m = 0; m < NC; m++) o[(size_t)m * cap + b] = val[m * R + rr];
      }
    }
    __syncthreads();
  }
  if (DIRECT) ext_fold_lf(lx, ly, sc->lf[f]);
}

void ext_prepare() {
  cudaFuncSetAttribute(k_ext_blocked<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ext_blocked_smem(4, SIF_EXT_BLOCKED_MAX));
  cudaFuncSetAttribute(k_ext_blocked<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ext_blocked_smem(2, SIF_EXT_BLOCKED_MAX));
  cudaGetLastError();
}

void launch_ext_blocked(const Grid &g, double *const wN[4], double *const wP[4], double *ul0,
                        double *ul1, int f0, int nf, const ExtPlan *plan, int cap,
                        const int *etiles, const int *nband, const int *map, const int *band,
                        int work, double *tmp, const double *alpha,
                        const unsigned char *const nostate[2], Scalars *sc, int num_sms,
                        cudaStream_t st) {
  ExtFields F;
  for (int m = 0; m < 4; m++) {
    F.p[0][m] = wN[m];
    F.p[1][m] = wP[m];
    F.p[2][m] = m == 0 ? ul0 : (m == 1 ? ul1 : nullptr);
  }
  F.ncomp[0] = F.ncomp[1] = 4;
  F.ncomp[2] = 2;
  for (int k = 0; k < 2; k++) {
    F.gamma[k] = g.gamma[k];
    F.pinf[k] = g.pinf[k];
  }
  // about one CTA per band tile (the CTAs loop over the device's tile
  // count): a band tile holds some 32 band cells or more, and a CTA that
  // finds no tile still takes a whole SM's registers to start
  int gx = ext_tiles(g);
  if (gx > work / 32 + 1) gx = work / 32 + 1;
  if (gx > 2 * num_sms) gx = 2 * num_sms;
  dim3 grid(gx, nf);
  if (f0 < 2) {
    // the stencil states' band values are in tmp (k_ext_setup's copy)
    launch_k(k_ext_blocked<4, true>, grid, EXT_THREADS, ext_blocked_smem(4, g.ext_iters), st, 
        g, F, f0, plan, cap, etiles, nband, map, tmp, nullptr, alpha, nostate[0], nostate[1],
        sc);
    sif_note_launches(1);
    return;
  }
  launch_k(k_ext_blocked<2, false>, grid, EXT_THREADS, ext_blocked_smem(2, g.ext_iters), st, 
      g, F, f0, plan, cap, etiles, nband, map, nullptr, tmp, alpha, nostate[0], nostate[1], sc);
  launch_k(k_ext_scatter, dim3(blocks_for(work, 64), nf), 64, 0, st, g, F, f0, cap, band, nband, tmp,
                                                               alpha, nostate[0], nostate[1], sc);
  sif_note_launches(2);
}

// ---------------------------------------------------------------------
// small-cell mixing with source plans (gather in the CPU reference's
// scatter order: sources in raster order, each adding to itself and
// subtracting at its targets)

__device__ bool mix_source_plan(const Grid &g, int k, int i, int j, const double *alpha,
                                const double *phi, double *const q[4], MixPlan &s) {
  int c = gidx(g, i, j);
  double as = vol_k(alpha, k, c);
  s.nt = 0;
  if (as >= g.mix_alpha) return false;
  // an empty small cell with no content has nothing to mix (q == nullptr:
  // the linearised mixing of the adjoint, which mixes it like any other)
  if (q && as == 0.0 && q[0][c] == 0.0 && q[1][c] == 0.0 && q[2][c] == 0.0 && q[3][c] == 0.0)
    return false;
  double nxv, nyv;
  unit_normal(g, phi, i, j, nxv, nyv);
  if (k == 0) {
    nxv = -nxv;
    nyv = -nyv;
  }
  int sx = nxv >= 0.0 ? 1 : -1, sy = nyv >= 0.0 ? 1 : -1;
  int ti[3] = {i + sx, i, i + sx}, tj[3] = {j, j + sy, j + sy};
  double wt[3] = {nxv * nxv, nyv * nyv, fabs(nxv * nyv)};
  int nt = g.dim == 2 ? 3 : 1;
  // targets: the normal-direction neighbours that are not small cells;
  // else the largest of the eight neighbours if it is not small; else the
  // normal-direction neighbours larger than the source
  bool keep[3] = {false, false, false};
  double sum = 0.0;
  for (int t = 0; t < nt; t++) {
    if (!inside(g, ti[t], tj[t]) || !(wt[t] > 0.0)) continue;
    if (!(vol_k(alpha, k, gidx(g, ti[t], tj[t])) >= g.mix_alpha)) continue;
    keep[t] = true;
    sum += wt[t];
  }
  s.as = as;
  if (!(sum > 0.0)) {
    int best = -1;
    double ab = 0.0;
    for (int dj = -1; dj <= 1; dj++)
      for (int di = -1; di <= 1; di++) {
        if ((di == 0 && dj == 0) || (g.dim == 1 && dj != 0) || !inside(g, i + di, j + dj))
          continue;
        double at = vol_k(alpha, k, gidx(g, i + di, j + dj));
        if (at > ab) {
          ab = at;
          best = gidx(g, i + di, j + dj);
        }
      }
    if (best >= 0 && ab >= g.mix_alpha) {
      s.tc[0] = best;
      s.beta[0] = 1.0;
      s.at[0] = ab;
      s.nt = 1;
      return true;
    }
    for (int t = 0; t < nt; t++) {
      if (!inside(g, ti[t], tj[t]) || !(wt[t] > 0.0)) continue;
      if (!(vol_k(alpha, k, gidx(g, ti[t], tj[t])) > as)) continue;
      keep[t] = true;
      sum += wt[t];
    }
  }
  if (!(sum > 0.0)) return false;
  for (int t = 0; t < nt; t++) {
    if (!keep[t]) continue;
    int tc = gidx(g, ti[t], tj[t]);
    s.tc[s.nt] = tc;
    s.beta[s.nt] = wt[t] / sum;
    s.at[s.nt] = vol_k(alpha, k, tc);
    s.nt++;
  }
  return true;
}

struct MixQ {
  double *q[2][4];
};

// One source's plan for a state-carrying fluid, written straight to its
// slot: the decisions and arithmetic of mix_source_plan, with the loads
// taken in two batches (the 3 x 3 volume fractions, the level set's face
// neighbours and the cell's state together, then the targets' states) and
// every array indexed at compile time so that it stays in registers.  Only
// what k_mix_apply reads is stored: the target count, the targets and the
// amounts.  Every index lies in the padded planes; inside() decides what
// is used.
__device__ void mix_setup_one(const Grid &g, int k, int i, int j, const double *alpha,
                              const double *phi, double *const q[4], MixPlan *out) {
  const int c = gidx(g, i, j);
  double a9[9];
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const int di = e % 3 - 1, dj = e / 3 - 1;
    a9[e] = (g.dim == 2 || dj == 0) ? vol_k(alpha, k, gidx(g, i + di, j + dj)) : 0.0;
  }
  const double pe = phi[gidx(g, i + 1, j)], pw = phi[gidx(g, i - 1, j)];
  const double pn = g.dim == 2 ? phi[gidx(g, i, j + 1)] : 0.0;
  const double ps = g.dim == 2 ? phi[gidx(g, i, j - 1)] : 0.0;
  double qs[4];
#pragma unroll
  for (int m = 0; m < 4; m++) qs[m] = q[m][c];
  const double as = a9[4];
  if (as >= g.mix_alpha || (as == 0.0 && qs[0] == 0.0 && qs[1] == 0.0 && qs[2] == 0.0 &&
                            qs[3] == 0.0)) {
    out->nt = 0;
    return;
  }
  // unit_normal's arithmetic on the loaded values, turned to point out of
  // fluid k
  double nxv = 0.0, nyv = 0.0;
  {
    const double gx = (pe - pw) / (2.0 * g.dx);
    const double gy = g.dim == 2 ? (pn - ps) / (2.0 * g.dy) : 0.0;
    const double m = sqrt(gx * gx + gy * gy);
    if (m > 0.0) {
      nxv = gx / m;
      nyv = gy / m;
    }
  }
  if (k == 0) {
    nxv = -nxv;
    nyv = -nyv;
  }
  const int sx = nxv >= 0.0 ? 1 : -1, sy = nyv >= 0.0 ? 1 : -1;
  // the normal-direction neighbours: across x, across y, the diagonal
  const int ti[3] = {i + sx, i, i + sx}, tj[3] = {j, j + sy, j + sy};
  const double at3[3] = {sx > 0 ? a9[5] : a9[3], sy > 0 ? a9[7] : a9[1],
                         sy > 0 ? (sx > 0 ? a9[8] : a9[6]) : (sx > 0 ? a9[2] : a9[0])};
  const double wt[3] = {nxv * nxv, nyv * nyv, fabs(nxv * nyv)};
  const int nt = g.dim == 2 ? 3 : 1;
  bool keep[3];
  double sum = 0.0;
#pragma unroll
  for (int t = 0; t < 3; t++) {
    keep[t] = t < nt && inside(g, ti[t], tj[t]) && wt[t] > 0.0 && at3[t] >= g.mix_alpha;
    if (keep[t]) sum += wt[t];
  }
  bool single = false;
  int best = -1;
  double ab = 0.0;
  if (!(sum > 0.0)) {
    // the largest of the eight neighbours (the first in raster order)
#pragma unroll
    for (int e = 0; e < 9; e++) {
      const int di = e % 3 - 1, dj = e / 3 - 1;
      if (e == 4 || (g.dim == 1 && dj != 0) || !inside(g, i + di, j + dj)) continue;
      if (a9[e] > ab) {
        ab = a9[e];
        best = e;
      }
    }
    if (best >= 0 && ab >= g.mix_alpha) {
      single = true;
    } else {
      // the normal-direction neighbours larger than the source
#pragma unroll
      for (int t = 0; t < 3; t++) {
        keep[t] = t < nt && inside(g, ti[t], tj[t]) && wt[t] > 0.0 && at3[t] > as;
        if (keep[t]) sum += wt[t];
      }
      if (!(sum > 0.0)) {
        out->nt = 0;
        return;
      }
    }
  }
  const int bestc = single ? gidx(g, i + best % 3 - 1, j + best / 3 - 1) : 0;
  bool use[3];
  int tcs[3];
  double bet[3], ats[3], qt[3][4];
#pragma unroll
  for (int t = 0; t < 3; t++) {
    use[t] = single ? t == 0 : keep[t];
    tcs[t] = single ? bestc : gidx(g, ti[t], tj[t]);
    bet[t] = single ? 1.0 : wt[t] / sum;
    ats[t] = single ? ab : at3[t];
#pragma unroll
    for (int m = 0; m < 4; m++) qt[t][m] = use[t] ? q[m][tcs[t]] : 0.0;
  }
  // M = beta (q_t as - q_s at) / (as beta + at), one division per target
  int p = 0;
#pragma unroll
  for (int t = 0; t < 3; t++) {
    if (!use[t]) continue;
    const double bd = bet[t] / (as * bet[t] + ats[t]);
    out->tc[p] = tcs[t];
#pragma unroll
    for (int m = 0; m < 4; m++) out->M[p][m] = (qt[t][m] * as - qs[m] * ats[t]) * bd;
    p++;
  }
  out->nt = p;
}

// plan of every band cell as a source, with the amounts it exchanges with
// its targets, M = beta (q_t as - q_s at) / (as beta + at) (as the product
// of the difference and beta / (as beta + at)), computed from the states
// before mixing
__global__ void k_mix_setup(Grid g, int mask, MixQ Q, const double *__restrict__ alpha,
                            const double *__restrict__ phi, const int *__restrict__ band,
                            const int *nband, MixPlan *plan, int cap) {
  SIF_TICK();
  const int k = blockIdx.y;  // fluid
  if (!(mask & (1 << k))) return;
  int n = *nband;
  // the fluid's planes chosen by select, not by a runtime index into the
  // parameter block (which would copy it to local memory)
  double *q[4];
#pragma unroll
  for (int m = 0; m < 4; m++) q[m] = k ? Q.q[1][m] : Q.q[0][m];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    mix_setup_one(g, k, i, j, alpha, phi, q, plan + (size_t)k * cap + idx);
  }
}

// each band cell adds what it receives as a source and subtracts what it
// gives as a target, in the CPU reference's scatter order (sources in
// raster order, targets in plan order).  A cell reads only its own state
// and the plans, so the update is written in place.
__global__ void k_mix_apply(Grid g, int mask, MixQ Q, const int *__restrict__ map,
                            const MixPlan *__restrict__ plan, int cap,
                            const int *__restrict__ band, const int *nband) {
  SIF_TICK();
  int k = blockIdx.y;
  if (!(mask & (1 << k))) return;
  int n = *nband;
  double *q[4];
#pragma unroll
  for (int m = 0; m < 4; m++) q[m] = k ? Q.q[1][m] : Q.q[0][m];
  const MixPlan *P = plan + (size_t)k * cap;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    // the neighbours' plan positions and target counts, loaded together
    int ps[9], nts[9];
#pragma unroll
    for (int e = 0; e < 9; e++) {
      int di = e % 3 - 1, dj = e / 3 - 1;
      bool ok = (g.dim == 2 || dj == 0) && inside(g, i + di, j + dj);
      ps[e] = ok ? map[gidx(g, i + di, j + dj)] : -1;
    }
#pragma unroll
    for (int e = 0; e < 9; e++) nts[e] = ps[e] >= 0 ? P[ps[e]].nt : 0;
    double val[4] = {q[0][c], q[1][c], q[2][c], q[3][c]};
#pragma unroll
    for (int e = 0; e < 9; e++) {
      if (!nts[e]) continue;
      const MixPlan &sp = P[ps[e]];
      bool self = e == 4;
      for (int t = 0; t < nts[e]; t++) {
        bool tgt = sp.tc[t] == c;
        if (!self && !tgt) continue;
        for (int m = 0; m < 4; m++) {
          if (self) val[m] += sp.M[t][m];
          if (tgt) val[m] -= sp.M[t][m];
        }
      }
    }
    for (int m = 0; m < 4; m++) q[m][c] = val[m];
  }
}

__global__ void k_mix_scatter(int mask, MixQ Q, const int *__restrict__ band, const int *nband,
                              const double *tmp) {
  SIF_TICK();
  int k = blockIdx.y;
  if (!(mask & (1 << k))) return;
  int n = *nband;
  const double *in = tmp + (size_t)k * 4 * n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    for (int m = 0; m < 4; m++) Q.q[k][m][c] = in[(size_t)m * n + idx];
  }
}

void launch_mix2(const Grid &g, int mask, double *const qN[4], double *const qP[4],
                 const double *alpha, const double *phi, const int *band, const int *map,
                 const int *nband, MixPlan *plan, int cap, int work, double *tmp,
                 cudaStream_t st) {
  MixQ Q;
  for (int m = 0; m < 4; m++) {
    Q.q[0][m] = qN ? qN[m] : nullptr;
    Q.q[1][m] = qP ? qP[m] : nullptr;
  }
  // small blocks spread the band's few thousand cells over the SMs
  int b = blocks_for(work, 64);
  launch_k(k_mix_setup, dim3(b, 2), 64, 0, st, g, mask, Q, alpha, phi, band, nband, plan, cap);
  launch_k(k_mix_apply, dim3(b, 2), 64, 0, st, g, mask, Q, map, plan, cap, band, nband);
  sif_note_launches(2);
}

// ---------------------------------------------------------------------
// transpose of the small-cell mixing (the adjoint of a frozen step): each
// source-target pair moved M = beta (q_t as - q_s at) / den from the
// target to the source, so the adjoint of the old states picks up
// (lam_s - lam_t) dM/dq.  Gathered per band cell like the forward.

__global__ void k_mix_adj_setup(Grid g, const double *__restrict__ alpha,
                                const double *__restrict__ phi, const int *__restrict__ band,
                                const int *nband, MixPlan *plan, int cap) {
  SIF_TICK();
  int n = *nband;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    for (int k = 0; k < 2; k++) {
      MixPlan s;
      mix_source_plan(g, k, i, j, alpha, phi, nullptr, s);
      plan[(size_t)k * cap + idx] = s;
    }
  }
}

__global__ void k_mix_adj_apply(Grid g, MixQ L, const int *__restrict__ map,
                                const MixPlan *__restrict__ plan, int cap,
                                const int *__restrict__ band, const int *nband, double *tmp) {
  SIF_TICK();
  int k = blockIdx.y;
  int n = *nband;
  double *const *lam = L.q[k];
  const MixPlan *P = plan + (size_t)k * cap;
  double *out = tmp + (size_t)k * 4 * n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    double val[4] = {lam[0][c], lam[1][c], lam[2][c], lam[3][c]};
    for (int dj = -1; dj <= 1; dj++) {
      if (g.dim == 1 && dj != 0) continue;
      for (int di = -1; di <= 1; di++) {
        if (!inside(g, i + di, j + dj)) continue;
        int s = gidx(g, i + di, j + dj);
        int ps = map[s];
        if (ps < 0) continue;
        const MixPlan &sp = P[ps];
        for (int t = 0; t < sp.nt; t++) {
          int tc = sp.tc[t];
          bool self = (s == c), tgt = (tc == c);
          if (!self && !tgt) continue;
          double den = sp.as * sp.beta[t] + sp.at[t];
          for (int m = 0; m < 4; m++) {
            double dM = lam[m][s] - lam[m][tc];
            if (self) val[m] -= dM * sp.beta[t] * sp.at[t] / den;
            if (tgt) val[m] += dM * sp.beta[t] * sp.as / den;
          }
        }
      }
    }
    for (int m = 0; m < 4; m++) out[(size_t)m * n + idx] = val[m];
  }
}

void launch_mix_adjoint(const Grid &g, double *const lN[4], double *const lP[4],
                        const double *alpha, const double *phi, const int *band, const int *map,
                        const int *nband, MixPlan *plan, int cap, int work, double *tmp,
                        cudaStream_t st) {
  MixQ L;
  for (int m = 0; m < 4; m++) {
    L.q[0][m] = lN[m];
    L.q[1][m] = lP[m];
  }
  int b = blocks_for(work, 128);
  launch_k(k_mix_adj_setup, b, 128, 0, st, g, alpha, phi, band, nband, plan, cap);
  launch_k(k_mix_adj_apply, dim3(b, 2), 128, 0, st, g, L, map, plan, cap, band, nband, tmp);
  launch_k(k_mix_scatter, dim3(b, 2), 128, 0, st, 3, L, band, nband, tmp);
  sif_note_launches(3);
}

SIF_TU_LAUNCH_READER(plan)
