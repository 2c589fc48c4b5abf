// FP64 roofline denominator: the device's fused multiply-add issue rate for
// double precision, measured with eight independent dependency chains per
// thread on every SM.  The result sink is a file-scope device variable, so the
// measurement allocates no memory.
#include <cuda_runtime.h>

#include "tde_internal.cuh"

namespace tde {

__device__ double g_peak_sink;

__global__ void k_dfma_chains(int iters, double seed) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + 1e-9 * (threadIdx.x + c);
  const double b = 0.999999999, cc = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, cc);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == 12345.678) g_peak_sink = s;  // keeps the chains live
}

}  // namespace tde

extern "C" int tde_measure_fp64_peak(double* fma_per_s) {
  using namespace tde;
  if (fma_per_s == nullptr) return TDE_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TDE_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TDE_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 2048;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TDE_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) return TDE_ECUDA;
  k_dfma_chains<<<blocks, threads>>>(64, 1.0);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_dfma_chains<<<blocks, threads>>>(iters, 1.0 + rep);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return TDE_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *fma_per_s = double(blocks) * threads * iters * 8.0 / (double(best) * 1e-3);
  return TDE_OK;
}
