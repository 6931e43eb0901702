// Arithmetic issue-rate probe: the roofline denominator for kernels bound by
// the FP64 (or FP32) pipes, measured on the GPU the solver runs on.  Each
// thread runs 8 independent FMA chains on registers; the grid fills every SM.
#include <cuda_runtime.h>

#include "sphere_poisson.h"

namespace {

template <typename T>
__global__ void k_fma_chains(T* out, T a, T b, int iters) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never taken; keeps the chains live
}

template <typename T>
int rate(int iters, double* gops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SP_ERR_CUDA;
  const int blocks = sms * 4, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return SP_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 2; ++w) k_fma_chains<T><<<blocks, threads>>>(out, (T)0.999999, (T)1e-7, iters);
  cudaEventRecord(e0);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, threads>>>(out, (T)0.999999, (T)1e-7, iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return SP_ERR_CUDA;
  *gops = (double)blocks * threads * iters * 8.0 * reps / (ms * 1e-3) * 1e-9;
  return SP_OK;
}

}  // namespace

extern "C" int sphere_poisson_pipe_rates(double* fp64_fma_gops, double* fp32_fma_gops) {
  if (!fp64_fma_gops || !fp32_fma_gops) return SP_ERR_NULL;
  int rc = rate<double>(2048, fp64_fma_gops);
  if (rc != SP_OK) return rc;
  return rate<float>(65536, fp32_fma_gops);
}
