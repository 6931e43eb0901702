// FP64 transform and elimination kernels (and the FP64 zonal side path of the FP32 forms).
#define SP_FP64_KERNELS
#include <algorithm>
#include "launchers.inl"
#include "batched.cuh"

namespace sp {

template <>
void launch_rows_forward<double>(bool adj, bool big, const Launch& l, const double* f, cpx<double>* W, int nt,
                                 int n, int Kp, int rows, const FftDesc& d, const cpx<double>* tw,
                                 const int* perm, const cpx<double>* post, const double* row_scale,
                                 const double* row_scale_t, cpx<double>* zonal) {
  SP_PICK(k_rows_forward, double, adj, big, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_rows_inverse<double>(bool adj, bool big, const Launch& l, const cpx<double>* W, double* u, int nt,
                                 int n, int Kp, int rows, const FftDesc& d, const cpx<double>* tw,
                                 const int* perm, const cpx<double>* post, const double* row_scale,
                                 const double* row_scale_t, const cpx<double>* zonal) {
  SP_PICK(k_rows_inverse, double, adj, big, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_theta_forward<double>(bool adj, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                                  int cols, const FftDesc& d, const cpx<double>* tw, const int* perm,
                                  const cpx<double>* post, double inv_n, int zonal) {
  SP_PICK(k_theta_forward, double, adj, big, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
void launch_theta_inverse<double>(bool adj, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                                  int cols, const FftDesc& d, const cpx<double>* tw, const int* perm,
                                  const cpx<double>* post, double inv_n, int zonal) {
  SP_PICK(k_theta_inverse, double, adj, big, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
cudaError_t allow_transform_smem<double>(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto upd = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  upd(cudaFuncSetAttribute(k_rows_forward<double, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<double, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<double, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward<double, true, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<double, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<double, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<double, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse<double, true, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<double, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<double, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<double, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward<double, true, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<double, false, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<double, false, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<double, true, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse<double, true, true>, a, bytes));
  upd(allow_pipe_smem<double>(bytes));
  return e;
}
template <>
void launch_solve<double>(bool adj, const Launch& l, cpx<double>* W, const double* fl, const double* fiu,
                          const double* fcu, int N, int K, int Kp) {
  if (adj) k_solve<true, double><<<l.grid, l.threads, l.smem, l.stream>>>(W, fl, fiu, fcu, N, K, Kp);
  else k_solve<false, double><<<l.grid, l.threads, l.smem, l.stream>>>(W, fl, fiu, fcu, N, K, Kp);
}
template <>
void launch_factor<double>(const Launch& l, double* fl, double* fiu, double* fcu, int N, int K, int Kp) {
  k_factor<double><<<l.grid, l.threads, l.smem, l.stream>>>(fl, fiu, fcu, N, K, Kp);
}

void launch_zonal_scan(bool adj, cudaStream_t st, cpx<double>* Z, const double* zl, const double* ziu,
                       const double* zcu, int N) {
  const int threads = 512;
  const size_t smem = threads * sizeof(AffineC);
  if (adj) k_zonal_scan<true><<<1, threads, smem, st>>>(Z, zl, ziu, zcu, N);
  else k_zonal_scan<false><<<1, threads, smem, st>>>(Z, zl, ziu, zcu, N);
}

cudaError_t batched_fp64_occupancy(bool big, int threads, size_t smem, int* blocks_per_sm) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if (big) {
    e = cudaFuncSetAttribute(k_batched_fp64<true>, a, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batched_fp64<true>, threads, smem);
  } else {
    e = cudaFuncSetAttribute(k_batched_fp64<false>, a, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batched_fp64<false>, threads, smem);
  }
  return e;
}
void launch_batched_fp64(bool big, dim3 grid, int threads, size_t smem, cudaStream_t st, const BatchArgs& a) {
  if (big) k_batched_fp64<true><<<grid, threads, smem, st>>>(a);
  else k_batched_fp64<false><<<grid, threads, smem, st>>>(a);
}

void launch_sum2_finish(cudaStream_t st, const cpx<double>* C, int N, int Kp, double* out) {
  k_sum2_finish<<<1, 256, 0, st>>>(C, N, Kp, out);
}
void launch_msin_div(cudaStream_t st, const cpx<double>* X, cpx<double>* Q, int N, int K, int Kp) {
  const int threads = 128;
  k_msin_div<<<(2 * Kp + threads - 1) / threads, threads, 0, st>>>(X, Q, N, K, Kp);
}
void launch_tangential(cudaStream_t st, const cpx<double>* X, const cpx<double>* Q, cpx<double>* G, int N, int K,
                       int Kp, int comp) {
  const int threads = 256;
  const size_t total = (size_t)N * Kp;
  k_tangential<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(X, Q, G, N, K, Kp, comp);
}

void launch_ge_pivot(cudaStream_t st, const double* e, int nt, int n, GePivot* part, int nparts, GePivot* out) {
  k_ge_pivot_partial<<<nparts, 256, 0, st>>>(e, nt, n, part);
  k_ge_pivot_final<<<1, 1, 0, st>>>(e, n, part, nparts, out);
}
void launch_ge_step(cudaStream_t st, double* e, int nt, int n, int istar, int qstar, double* col, double* row,
                    double p0, double p1, size_t total) {
  const int threads = 256;
  const int ext = std::max(2 * nt, n);
  k_ge_extract<<<(ext + threads - 1) / threads, threads, 0, st>>>(e, nt, n, istar, qstar, col, row);
  k_ge_update<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(e, nt, n, col, row, p0, p1);
}
void launch_lowrank_pack(cudaStream_t st, const double* cols, int terms, int nt, const double* sin2, cpx<double>* Wc) {
  const int threads = 256, total = nt * terms;
  k_lowrank_pack<<<(total + threads - 1) / threads, threads, 0, st>>>(cols, terms, nt, sin2, Wc);
}
void launch_lowrank_outer(cudaStream_t st, cpx<double>* Wc, const cpx<double>* R, const double* piv,
                          int terms, int N, int K, int Kp, cpx<double>* F) {
  const int threads = 256;
  if (terms > 0) k_lowrank_weights<<<(N * terms + threads - 1) / threads, threads, 0, st>>>(Wc, piv, terms, N);
  const dim3 grid((Kp + threads - 1) / threads, N);
  k_lowrank_outer<<<grid, threads, (size_t)2 * terms * sizeof(cpx<double>), st>>>(Wc, R, terms, K, Kp, F);
}

SP_INSTANTIATE_PIPE(double);

}  // namespace sp
