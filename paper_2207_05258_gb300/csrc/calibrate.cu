// Measured ceiling of the FP64 pipe: a loop of independent DFMA chains (no
// memory traffic, no dependence between the chains of a thread), eight warps
// per SM. The stencil kernels are FP64-pipe bound; this gives the rate that
// plain DFMA work reaches on the device at its current clocks, next to the
// nominal figure (2 DFMA per clock per SM).
#include <cuda_runtime.h>

#include "hweno.h"

namespace hweno {
namespace {

constexpr int kChains = 8, kIters = 4096, kThreads = 128, kCtasPerSm = 2;

__global__ void __launch_bounds__(kThreads) k_dfma_loop(double* out, double m, double c) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the loop
}

}  // namespace
}  // namespace hweno

extern "C" int hweno_measure_fp64_peak(double* tflops, void* stream) {
  using namespace hweno;
  if (!tflops) return HWENO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HWENO_ECUDA;
  const int blocks = sms * kCtasPerSm;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * kThreads) != cudaSuccess) return HWENO_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HWENO_OK;
  float best = 1e30f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = HWENO_ECUDA;
  } else {
    for (int r = 0; r < 6 && rc == HWENO_OK; ++r) {  // the first launch warms up
      cudaEventRecord(e0, s);
      k_dfma_loop<<<blocks, kThreads, 0, s>>>(out, 0.999999, 1e-7);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = HWENO_ECUDA;
      else if (r > 0 && ms < best)
        best = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != HWENO_OK) return rc;
  const double dfma = (double)blocks * kThreads * kIters * kChains;
  *tflops = 2.0 * dfma / (best * 1e-3) / 1e12;
  return HWENO_OK;
}
