// FP64 transform and elimination kernels (and the FP64 zonal side path of the
// FP32 forms), and the FP64 operators of calculus.cuh.
#include <algorithm>
#include "launchers.inl"
#include "batched.cuh"
#include "calculus.cuh"
#include "poles.cuh"

namespace sp {

// FP64 transforms whose passes all have scaled twiddle records run in the
// kernels bounded to two 512-thread CTAs per SM (the *_two kernels)
static bool two_ctas(const FftDesc& d) {
  for (int s = 0; s < d.nstages; ++s) {
    const int r = d.radix[s];
    if (r != 2 && r != 3 && r != 4 && r != 5 && r != 8) return false;
  }
  return true;
}

#define SP_PICK64(FN, ADJV, BIGV, DESC, ...)                                                   \
  do {                                                                                         \
    if (!(BIGV) && two_ctas(DESC)) {                                                           \
      if (ADJV) FN##_two<double, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);  \
      else FN##_two<double, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);      \
    } else {                                                                                   \
      SP_PICK(FN, double, ADJV, BIGV, __VA_ARGS__);                                            \
    }                                                                                          \
  } while (0)

template <>
void launch_rows_forward<double>(bool adj, bool big, const Launch& l, const double* f, cpx<double>* W, int nt,
                                 int n, int Kp, int rows, const FftDesc& d, const cpx<double>* tw,
                                 const int* perm, const cpx<double>* post, const double* row_scale,
                                 const double* row_scale_t, cpx<double>* zonal) {
  SP_PICK64(k_rows_forward, adj, big, d, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_rows_inverse<double>(bool adj, bool big, const Launch& l, const cpx<double>* W, double* u, int nt,
                                 int n, int Kp, int rows, const FftDesc& d, const cpx<double>* tw,
                                 const int* perm, const cpx<double>* post, const double* row_scale,
                                 const double* row_scale_t, const cpx<double>* zonal) {
  SP_PICK64(k_rows_inverse, adj, big, d, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <>
void launch_theta_forward<double>(bool adj, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                                  int cols, const FftDesc& d, const cpx<double>* tw, const int* perm,
                                  const cpx<double>* post, double inv_n, int zonal) {
  SP_PICK64(k_theta_forward, adj, big, d, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <>
void launch_theta_inverse<double>(bool adj, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                                  int cols, const FftDesc& d, const cpx<double>* tw, const int* perm,
                                  const cpx<double>* post, double inv_n, int zonal) {
  SP_PICK64(k_theta_inverse, adj, big, d, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
void launch_theta_poles_adj(bool last, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                            const FftDesc& d, const cpx<double>* tw, const int* perm) {
  if (last) {
    if (big) k_theta_poles_adj_last<true><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
    else k_theta_poles_adj_last<false><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
  } else {
    if (big) k_theta_poles_adj_first<true><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
    else k_theta_poles_adj_first<false><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
  }
}
void launch_theta_poles(bool inverse, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                        const FftDesc& d, const cpx<double>* tw, const int* perm) {
  if (inverse) {
    if (big) k_theta_inverse_poles<true><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
    else k_theta_inverse_poles<false><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
  } else {
    if (big) k_theta_forward_poles<true><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
    else k_theta_forward_poles<false><<<l.grid, l.threads, l.smem, l.stream>>>(W, N, K, Kp, d, tw, perm);
  }
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
  upd(cudaFuncSetAttribute(k_theta_forward_poles<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward_poles<true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse_poles<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse_poles<true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_poles_adj_first<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_poles_adj_first<true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_poles_adj_last<false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_poles_adj_last<true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward_two<double, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_forward_two<double, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse_two<double, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse_two<double, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward_two<double, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward_two<double, true>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse_two<double, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse_two<double, true>, a, bytes));
  upd(allow_pipe_smem<double>(bytes));
  return e;
}
template <>
void launch_solve<double>(bool adj, const Launch& l, cpx<double>* W, const double* fl, const double* fiu,
                          const double* fcu, int N, int K, int Kp) {
  // two warps per CTA (the twisted solve); l.threads is not used
  if (adj) k_solve<true, double><<<l.grid, kSolveThreads, 0, l.stream>>>(W, fl, fiu, fcu, N, K, Kp);
  else k_solve<false, double><<<l.grid, kSolveThreads, 0, l.stream>>>(W, fl, fiu, fcu, N, K, Kp);
}
template <>
void launch_factor<double>(const Launch& l, double* fl, double* fiu, double* fcu, int N, int K, int Kp, bool twist) {
  if (twist) k_factor<double, true><<<l.grid, l.threads, l.smem, l.stream>>>(fl, fiu, fcu, N, K, Kp);
  else k_factor<double, false><<<l.grid, l.threads, l.smem, l.stream>>>(fl, fiu, fcu, N, K, Kp);
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
void launch_mean(cudaStream_t st, const double* f, int nt, int n, const double* wrow, double2* part, int nparts,
                 double* mean, double* absmax) {
  k_mean_partial<<<nparts, 256, 0, st>>>(f, nt, n, wrow, part);
  k_mean_final<<<1, 256, 0, st>>>(part, nparts, mean, absmax);
}
size_t msin_scratch_bytes(int N, int Kp) {
  const size_t chunks = (size_t)(N + kMsinRows - 1) / kMsinRows;
  return 2 * chunks * (size_t)Kp * sizeof(cpx<double>);
}
void launch_msin_div(cudaStream_t st, const cpx<double>* X, cpx<double>* Q, cpx<double>* P, int N, int K, int Kp) {
  const int threads = 128, chunks = (N + kMsinRows - 1) / kMsinRows;
  const dim3 grid((Kp + threads - 1) / threads, chunks);
  k_msin_partial<<<grid, threads, 0, st>>>(X, P, N, K, Kp);
  k_msin_scan<<<(2 * Kp + threads - 1) / threads, threads, 0, st>>>(P, chunks, Kp);
  k_msin_apply<<<grid, threads, 0, st>>>(X, P, Q, N, K, Kp);
}
void launch_tangential(cudaStream_t st, const cpx<double>* X, const cpx<double>* Q, const TangentialCombo& tc,
                       int N, int K, int Kp) {
  const int threads = 128;
  const dim3 grid((Kp + threads - 1) / threads, std::min(N, 65535));
  switch (tc.acc & 7) {
    case 0: k_tangential<0><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    case 1: k_tangential<1><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    case 2: k_tangential<2><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    case 3: k_tangential<3><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    case 4: k_tangential<4><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    case 5: k_tangential<5><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    case 6: k_tangential<6><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
    default: k_tangential<7><<<grid, threads, 0, st>>>(X, Q, tc, N, K, Kp); break;
  }
}
void launch_coeff_chop(cudaStream_t st, cpx<double>* X, int N, int K, int Kp, unsigned long long* mx,
                       double rtol) {
  const int threads = 256;
  cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st);
  const dim3 grid((Kp + threads - 1) / threads, std::min(N, 128));
  k_coeff_absmax<<<grid, threads, 0, st>>>(X, N, K, Kp, mx);
  k_coeff_chop<<<grid, threads, 0, st>>>(X, N, K, Kp, mx, rtol);
}
namespace {
dim3 grid_points(int nt, int nl, int threads) {
  return dim3((nl + threads - 1) / threads, std::min(nt, 4096));
}
}  // namespace
void launch_cross_normal(cudaStream_t st, double* a, double* b, double* c, const double* geo, int nt, int nl) {
  const int threads = 256;
  k_cross_normal<<<grid_points(nt, nl, threads), threads, 0, st>>>(a, b, c, geo, nt, nl);
}
void launch_normal_dot(cudaStream_t st, const double* a, const double* b, const double* c, double* out,
                       const double* geo, int nt, int nl) {
  const int threads = 256;
  k_normal_dot<<<grid_points(nt, nl, threads), threads, 0, st>>>(a, b, c, out, geo, nt, nl);
}

void launch_ge_pivot(cudaStream_t st, const double* e, int nt, int n, GePivot* part, int nparts, GePivot* out) {
  k_ge_pivot_partial<<<nparts, 256, 0, st>>>(e, nt, n, part);
  k_ge_pivot_final<<<1, 256, 0, st>>>(e, n, part, nparts, out);
}
void launch_ge_step(cudaStream_t st, double* e, int nt, int n, int istar, int qstar, double* col, double* row,
                    double p0, double p1, double* AB) {
  const int threads = 256;
  const int ext = std::max(2 * nt, n);
  k_ge_extract<<<(ext + threads - 1) / threads, threads, 0, st>>>(e, nt, n, istar, qstar, col, row, p0, p1, AB);
  const dim3 grid((n + threads - 1) / threads, std::min(nt, 512));
  k_ge_update<<<grid, threads, 0, st>>>(e, nt, n, col, AB);
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
