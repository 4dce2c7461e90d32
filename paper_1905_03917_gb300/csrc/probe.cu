// probe.cu -- FP64 fused multiply-add throughput of the device: the
// arithmetic ceiling of the finite-volume kernel, which is bound by the
// FP64 pipe rather than by HBM bandwidth; and the finite-volume kernel's
// reciprocal over caller data, for tests against IEEE division.
#include "sif_internal.cuh"

// eight independent FMA chains per thread, ILP enough to fill the pipe
__global__ void k_dfma(double *out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
      x4 = fma(x4, a, b);
      x5 = fma(x5, a, b);
      x6 = fma(x6, a, b);
      x7 = fma(x7, a, b);
    }
  }
  double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == 1.2345) out[blockIdx.x] = s;  // keeps the chains live
}

extern "C" int sif_measure_fp64_peak(int device, double *tflops) {
  if (!tflops) return SIF_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return SIF_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * 65536) != cudaSuccess) return SIF_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8, iters = 2000;
  k_dfma<<<blocks, threads>>>(out, 50, 0.999999, 1e-7);  // warm-up
  cudaEventRecord(e0);
  k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.0f) return SIF_ECUDA;
  double flops = 2.0 * 8.0 * 16.0 * iters * (double)threads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SIF_OK;
}

__global__ void k_recip(const double *d, double *r, long long n) {
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += step)
    r[i] = recip_newton3(d[i]);
}

extern "C" int sif_probe_reciprocal(const double *d, double *r, long long n, void *stream) {
  if (n < 0 || (n > 0 && (!d || !r))) return SIF_EINVAL;
  if (n == 0) return SIF_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long want = (n + 255) / 256, cap = (long long)(sms > 0 ? sms : 1) * 8;
  int blocks = (int)(want < cap ? want : cap);
  k_recip<<<blocks, 256, 0, (cudaStream_t)stream>>>(d, r, n);
  return cudaGetLastError() == cudaSuccess ? SIF_OK : SIF_ECUDA;
}
