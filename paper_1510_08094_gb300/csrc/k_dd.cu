// Double-float transform kernels and the refinement kernels (the SP_FP32_REFINE form).
// That form has no adjoint, so only the forward instantiations exist.
#define SP_REFINE_KERNELS
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include "launchers.inl"
#include "fused_refine.cuh"

namespace sp {

template <>
void launch_rows_forward<dd>(bool adj, bool big, const Launch& l, const double* f, cpx<dd>* W, int nt, int n,
                             int Kp, int rows, const FftDesc& d, const cpx<dd>* tw, const int* perm,
                             const cpx<dd>* post, const double* row_scale, const dd* row_scale_t, cpx<double>* zonal) {
  (void)adj;
  SP_PICK_FWD(k_rows_forward, dd, big, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_rows_inverse<dd>(bool adj, bool big, const Launch& l, const cpx<dd>* W, double* u, int nt, int n,
                             int Kp, int rows, const FftDesc& d, const cpx<dd>* tw, const int* perm,
                             const cpx<dd>* post, const double* row_scale, const dd* row_scale_t, const cpx<double>* zonal) {
  (void)adj;
  SP_PICK_FWD(k_rows_inverse, dd, big, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_theta_forward<dd>(bool adj, bool big, const Launch& l, cpx<dd>* W, int N, int K, int Kp, int cols,
                              const FftDesc& d, const cpx<dd>* tw, const int* perm, const cpx<dd>* post,
                              dd inv_n, int zonal) {
  (void)adj;
  SP_PICK_FWD(k_theta_forward, dd, big, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
void launch_theta_inverse<dd>(bool adj, bool big, const Launch& l, cpx<dd>* W, int N, int K, int Kp, int cols,
                              const FftDesc& d, const cpx<dd>* tw, const int* perm, const cpx<dd>* post,
                              dd inv_n, int zonal) {
  (void)adj;
  SP_PICK_FWD(k_theta_inverse, dd, big, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
cudaError_t allow_transform_smem<dd>(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto upd = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  upd(cudaFuncSetAttribute(k_rows_forward<dd, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<dd, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<dd, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<dd, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<dd, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<dd, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<dd, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<dd, false, true>, a, bytes));
  upd(allow_pipe_smem<dd>(bytes));
  upd(cudaFuncSetAttribute(k_refine_fused<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_refine_fused<true>, a, bytes));
  return e;
}
namespace {
// the driver's tensor-map encoder, through the runtime (no link-time libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}
// the [N][Kp] double-float spectrum as a 2D array of 32-bit words (4 per
// element), box = one element (16 bytes) x kRefineBoxRows rows
bool encode_column_map(CUtensorMap* m, const cpx<dd>* W, int N, int Kp) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !W || N < 1 || (reinterpret_cast<uintptr_t>(W) & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)4 * Kp, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(cpx<dd>)};
  const cuuint32_t box[2] = {4, (cuuint32_t)kRefineBoxRows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<cpx<dd>*>(W), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void launch_refine_fused(bool big, const Launch& l, cpx<dd>* W, int N, int K, int Kp, const FftDesc& d,
                         const cpx<dd>* tw, const int* perm, const cpx<dd>* post_s, const cpx<dd>* post,
                         const float* fiu, int sweeps, int* status) {
  if (K < 2) return;   // column 0 only: nothing for this kernel
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const int use_tma = status && encode_column_map(&tm, W, N, Kp) ? 1 : 0;
  // persistent: as many CTAs as fit on the device at once, less one, at most one
  // per column.  A resident CTA fills its SM's registers and shared memory, so
  // the one SM left free is where the zonal column's one-CTA kernels (the
  // plan's high-priority side stream) run meanwhile instead of after the stage.
  int dev = 0, sms = 1, bps = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (big) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_refine_fused<true>, l.threads, l.smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_refine_fused<false>, l.threads, l.smem);
  const int resident = bps > 0 ? std::max(1, bps * sms - 1) : K - 1;
  const dim3 grid(std::min(K - 1, resident));
  if (big)
    k_refine_fused<true><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm, post_s, post, fiu, sweeps,
                                                                  tm, use_tma, status);
  else
    k_refine_fused<false><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm, post_s, post, fiu, sweeps,
                                                                   tm, use_tma, status);
}
size_t refine_fused_smem(int N, int threads) { return refine_fused_smem_bytes(N, threads); }

// one thread polls `polls` times for an mbarrier phase that nothing completes
// (no arrival, no copy in flight), then records kStatusTmaTimeout: the path a
// TMA wait takes when its copies never land
__global__ void k_wait_selftest(int* status, unsigned polls) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  mbar_init_fence();
  if (!mbar_wait_bounded(&bar, 0, polls)) atomicExch(status, kStatusTmaTimeout);
}
void launch_wait_selftest(int* status, unsigned polls, cudaStream_t st) {
  k_wait_selftest<<<1, 1, 0, st>>>(status, polls);
}

void launch_refine(const Launch& l, const cpx<dd>* F, cpx<dd>* X, cpx<float>* Y, const float* fl,
                   const float* fiu, const float* fcu, int N, int K, int Kp, int first) {
  // two warps per CTA (the twisted form); l.threads is not used
  k_refine<<<l.grid, kRefineThreads, 0, l.stream>>>(F, X, Y, fl, fiu, fcu, N, K, Kp, first);
}
void launch_zonal_extract(const Launch& l, const cpx<dd>* Wdd, cpx<double>* Z, int N, int Kp) {
  k_zonal_extract<<<l.grid, l.threads, l.smem, l.stream>>>(Wdd, Z, N, Kp);
}
void launch_zonal_insert(const Launch& l, const cpx<double>* Z, cpx<dd>* X, int N, int Kp) {
  k_zonal_insert<<<l.grid, l.threads, l.smem, l.stream>>>(Z, X, N, Kp);
}

SP_INSTANTIATE_PIPE(dd);

}  // namespace sp
