// FP32 transform and elimination kernels (the SP_FP32 form).
#include "launchers.inl"

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
  return e;
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
