// Persistent batched FP32 + refinement kernel (double-float transforms); its own
// translation unit so it compiles in parallel with the single-plan kernels.
#include "batched_dd.cuh"
#include "launch.h"

namespace sp {

cudaError_t batched_refine_occupancy(bool big, int threads, size_t smem, int* blocks_per_sm) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if (big) {
    e = cudaFuncSetAttribute(k_batched_refine<true>, a, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batched_refine<true>, threads, smem);
  } else {
    e = cudaFuncSetAttribute(k_batched_refine<false>, a, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batched_refine<false>, threads, smem);
  }
  return e;
}

void launch_batched_refine(bool big, dim3 grid, int threads, size_t smem, cudaStream_t st, const BatchArgs& a) {
  if (big) k_batched_refine<true><<<grid, threads, smem, st>>>(a);
  else k_batched_refine<false><<<grid, threads, smem, st>>>(a);
}

}  // namespace sp
