// FP32 transform and elimination kernels (the SP_FP32 form).
#include <cudaTypedefs.h>

#include <cstring>

#include "launchers.inl"
#include "fused.cuh"

namespace sp {

template <>
void launch_rows_forward<float>(bool adj, bool big, const Launch& l, const double* f, cpx<float>* W, int nt,
                                 int n, int Kp, int rows, const FftDesc& d, const cpx<float>* tw,
                                 const int* perm, const cpx<float>* post, const double* row_scale,
                                 const float* row_scale_t, cpx<double>* zonal) {
  SP_PICK(k_rows_forward, float, adj, big, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_rows_inverse<float>(bool adj, bool big, const Launch& l, const cpx<float>* W, double* u, int nt,
                                 int n, int Kp, int rows, const FftDesc& d, const cpx<float>* tw,
                                 const int* perm, const cpx<float>* post, const double* row_scale,
                                 const float* row_scale_t, const cpx<double>* zonal) {
  SP_PICK(k_rows_inverse, float, adj, big, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_theta_forward<float>(bool adj, bool big, const Launch& l, cpx<float>* W, int N, int K, int Kp,
                                  int cols, const FftDesc& d, const cpx<float>* tw, const int* perm,
                                  const cpx<float>* post, float inv_n, int zonal) {
  SP_PICK(k_theta_forward, float, adj, big, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
void launch_theta_inverse<float>(bool adj, bool big, const Launch& l, cpx<float>* W, int N, int K, int Kp,
                                  int cols, const FftDesc& d, const cpx<float>* tw, const int* perm,
                                  const cpx<float>* post, float inv_n, int zonal) {
  SP_PICK(k_theta_inverse, float, adj, big, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
cudaError_t allow_transform_smem<float>(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto upd = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  upd(cudaFuncSetAttribute(k_rows_forward<float, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<float, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<float, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<float, true, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<float, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<float, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<float, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<float, true, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<float, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<float, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<float, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<float, true, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<float, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<float, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<float, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<float, true, true>, a, bytes));
  upd(allow_pipe_smem<float>(bytes));
  upd(cudaFuncSetAttribute(k_theta_fused<float, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused<float, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused_cl<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused_cl<true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused1<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused1<true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused1_adj<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_fused1_adj<true>, a, bytes));
  return e;
}
namespace {
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
// the [N][Kp] FP32 spectrum as a 2D array of 32-bit words (2 per element),
// box = two elements (16 bytes) x kFusedBoxRows rows
bool encode_pair_map(CUtensorMap* m, const cpx<float>* W, int N, int Kp) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !W || N < 1 || (Kp & 1) || (reinterpret_cast<uintptr_t>(W) & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * Kp, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(cpx<float>)};
  const cuuint32_t box[2] = {4, (cuuint32_t)kFusedBoxRows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<cpx<float>*>(W), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void launch_theta_fused(bool big, const Launch& l, cpx<float>* W, int N, int K, int Kp, int cols, const FftDesc& d,
                        const cpx<float>* tw, const int* perm, const cpx<float>* post_s, const cpx<float>* post,
                        const float* fiu, float inv_n, int* status) {
  if (cols < 0) {    // the single-buffer form, -cols columns per CTA
    const int q = -cols;
    const dim3 grid((K + q - 1) / q);
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof(tm));
    const int use_tma =
        status && !big && fused1_tma_fits(N, q, l.threads) && encode_pair_map(&tm, W, N, Kp) ? 1 : 0;
    if (big)
      k_theta_fused1<true><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, q, d, tw, perm, post_s, post, fiu,
                                                                   tm, use_tma, status);
    else
      k_theta_fused1<false><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, q, d, tw, perm, post_s, post, fiu,
                                                                    tm, use_tma, status);
    return;
  }
  if (cols == 0) {   // the cluster form: one column per CTA, clusters of kFuseCluster
    const dim3 grid(((K + kFuseCluster - 1) / kFuseCluster) * kFuseCluster);
    if (big)
      k_theta_fused_cl<true><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm, post_s, post, fiu);
    else
      k_theta_fused_cl<false><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm, post_s, post, fiu);
    return;
  }
  if (big)
    k_theta_fused<float, true><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, cols, d, tw, perm, post_s,
                                                                        post, fiu, inv_n);
  else
    k_theta_fused<float, false><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, cols, d, tw, perm, post_s,
                                                                         post, fiu, inv_n);
}
void launch_theta_fused_adj(bool big, const Launch& l, cpx<float>* W, int N, int K, int Kp, int cols,
                            const FftDesc& d, const cpx<float>* tw, const int* perm, const cpx<float>* post,
                            const float* fiu, float inv_n, int* status) {
  const int q = cols < 0 ? -cols : 1;
  const dim3 grid((K + q - 1) / q);
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const int use_tma = status && !big && fused1_tma_fits(N, q, l.threads) && encode_pair_map(&tm, W, N, Kp) ? 1 : 0;
  if (big)
    k_theta_fused1_adj<true><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, q, d, tw, perm, post, fiu, inv_n,
                                                                     tm, use_tma, status);
  else
    k_theta_fused1_adj<false><<<grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, q, d, tw, perm, post, fiu, inv_n,
                                                                      tm, use_tma, status);
}
size_t theta_fused_smem(int N, int cols, int threads) {
  if (cols < 0) return fused1_smem_bytes(N, -cols, threads);
  return fused_smem_bytes<float>(N, cols > 0 ? cols : 1, threads);
}
void launch_factor_cols(const Launch& l, float* fiu, int N, int K) {
  k_factor_cols<float><<<l.grid, l.threads, l.smem, l.stream>>>(fiu, N, K);
}
template <>
void launch_solve<float>(bool adj, const Launch& l, cpx<float>* W, const float* fl, const float* fiu,
                         const float* fcu, int N, int K, int Kp) {
  // two warps per CTA (the twisted solve); l.threads is not used
  if (adj) k_solve<true, float><<<l.grid, kSolveThreads, 0, l.stream>>>(W, fl, fiu, fcu, N, K, Kp);
  else k_solve<false, float><<<l.grid, kSolveThreads, 0, l.stream>>>(W, fl, fiu, fcu, N, K, Kp);
}
template <>
void launch_factor<float>(const Launch& l, float* fl, float* fiu, float* fcu, int N, int K, int Kp, bool twist) {
  if (twist) k_factor<float, true><<<l.grid, l.threads, l.smem, l.stream>>>(fl, fiu, fcu, N, K, Kp);
  else k_factor<float, false><<<l.grid, l.threads, l.smem, l.stream>>>(fl, fiu, fcu, N, K, Kp);
}

SP_INSTANTIATE_PIPE(float);

}  // namespace sp
