// noalloc.cu -- conserved totals of caller-provided planes without any
// device allocation: the row partial sums live in a file-scope device array
// instead of context memory.
//
// Some callers cannot allocate device memory at the point where they need
// the totals: a host framework whose caching allocator has already claimed
// the GPU's free memory (a cudaMalloc would fail or fragment it), or a
// monitoring hook inside a time-stepping loop where an allocation would
// synchronise the device.  For them sif_integrals_noalloc works on planes
// they already own and writes into an output they already own.
#include <atomic>

#include "sif_internal.cuh"

// Scratch for the per-row partial sums of the 8 planes (8 * max rows
// doubles, 1 MiB).  Every process that loads the library holds this on
// each GPU it uses until it exits.
#define NOALLOC_MAX_ROWS 16384
static __device__ __align__(256) double g_noalloc_rows[8 * NOALLOC_MAX_ROWS];

struct NoallocPlanes {
  const double *p[8];
};

// one warp per row, lanes stride along x, then a fixed-order warp sum: the
// same summation order as the context reduction
__global__ void k_noalloc_rows(NoallocPlanes planes, int nx, int ny, double *rows) {
  int pl = blockIdx.y;
  const double *a = planes.p[pl];
  int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  double s = 0.0;
  if (j < ny)
    for (int i = lane; i < nx; i += 32) s += a[(size_t)j * nx + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0 && j < ny) rows[(size_t)pl * ny + j] = s;
}

__global__ void k_noalloc_final(const double *rows, int ny, double dxdy, double *out) {
  int pl = threadIdx.x;
  if (pl >= 8) return;
  double s = 0.0;
  for (int j = 0; j < ny; j++) s += rows[(size_t)pl * ny + j];
  out[pl] = s * dxdy;
}

// device address of the scratch array, looked up once per device (it is
// no longer valid after a cudaDeviceReset, which unloads the module).
// Concurrent first calls on one device store the same value; the atomics
// keep those stores well defined.
static std::atomic<void *> g_scratch_addr[64];

extern "C" int sif_integrals_noalloc(const double *q_N, const double *q_P, int nx, int ny,
                                     double dx, double dy, double *out, void *stream) {
  if (!q_N || !q_P || !out || nx < 1 || ny < 1) return SIF_EINVAL;
  if (ny > NOALLOC_MAX_ROWS) return SIF_EINVAL;  // scratch holds NOALLOC_MAX_ROWS rows
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SIF_ECUDA;
  void *ptr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    // set-up on the current device: the host-side name of the array is not
    // a device address, so ask the runtime for the address once
    if (cudaGetSymbolAddress(&ptr, g_noalloc_rows) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return SIF_ECUDA;
    }
    g_scratch_addr[dev].store(ptr, std::memory_order_release);
  }
  double *rows = (double *)ptr;
  cudaStream_t st = (cudaStream_t)stream;
  NoallocPlanes planes;
  for (int m = 0; m < 4; m++) {
    planes.p[m] = q_N + (size_t)m * nx * ny;
    planes.p[4 + m] = q_P + (size_t)m * nx * ny;
  }
  dim3 grid((ny + 7) / 8, 8);
  k_noalloc_rows<<<grid, 256, 0, st>>>(planes, nx, ny, rows);
  k_noalloc_final<<<1, 32, 0, st>>>(rows, ny, dx * dy, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIF_OK : SIF_ECUDA;
}
