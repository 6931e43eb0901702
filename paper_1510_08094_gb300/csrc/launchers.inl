// Definitions of the launchers declared in launch.h, included by the
// per-type translation units (the type's kernels are instantiated there).
#include "kernels.cuh"
#include "launch.h"

namespace sp {

#define SP_PICK(FN, T, ADJV, BIGV, ...)                                         \
  do {                                                                          \
    if (ADJV) {                                                                 \
      if (BIGV) FN<T, true, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);   \
      else FN<T, true, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);       \
    } else {                                                                    \
      if (BIGV) FN<T, false, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);  \
      else FN<T, false, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);      \
    }                                                                           \
  } while (0)

// forward-only types (the double-float form has no adjoint) instantiate ADJ = false only
#define SP_PICK_FWD(FN, T, BIGV, ...)                                           \
  do {                                                                          \
    if (BIGV) FN<T, false, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);    \
    else FN<T, false, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);        \
  } while (0)

// pipelined transform kernels (ADJ = false only for the forward-only double-float type)
#define SP_PIPE(FN, T, ADJV, ...)                                                          \
  do {                                                                                     \
    if constexpr (std::is_same<T, dd>::value) {                                            \
      FN<T, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);                   \
    } else {                                                                               \
      if (ADJV) FN<T, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);          \
      else FN<T, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);              \
    }                                                                                      \
  } while (0)

template <typename T>
void launch_rows_forward_pipe(bool adj, const Launch& l, const double* f, cpx<T>* W, int nt, int n, int Kp,
                              int rows, const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post,
                              const double* row_scale, const T* row_scale_t, cpx<double>* zonal) {
  SP_PIPE(k_rows_forward_pipe, T, adj, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <typename T>
void launch_rows_inverse_pipe(bool adj, const Launch& l, const cpx<T>* W, double* u, int nt, int n, int Kp,
                              int rows, const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post,
                              const double* row_scale, const T* row_scale_t, const cpx<double>* zonal) {
  SP_PIPE(k_rows_inverse_pipe, T, adj, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}
template <typename T>
void launch_theta_forward_pipe(bool adj, const Launch& l, cpx<T>* W, int N, int K, int Kp, int cols,
                               const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                               int zonal) {
  SP_PIPE(k_theta_forward_pipe, T, adj, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <typename T>
void launch_theta_inverse_pipe(bool adj, const Launch& l, cpx<T>* W, int N, int K, int Kp, int cols,
                               const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                               int zonal) {
  SP_PIPE(k_theta_inverse_pipe, T, adj, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}

// occupancy of a pipelined kernel (stage 0 rows_forward, 1 theta_forward, 2
// theta_inverse, 3 rows_inverse) with `smem` dynamic bytes (the kernels'
// shared-memory cap is raised once per device by allow_pipe_smem)
template <typename K>
cudaError_t occupancy_of(K kernel, int threads, size_t smem, int* bps) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kernel, threads, smem);
}
template <typename T>
cudaError_t allow_pipe_smem(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto upd = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  upd(cudaFuncSetAttribute(k_rows_forward_pipe<T, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_rows_inverse_pipe<T, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_forward_pipe<T, false>, a, bytes));
  upd(cudaFuncSetAttribute(k_theta_inverse_pipe<T, false>, a, bytes));
  if constexpr (!std::is_same<T, dd>::value) {
    upd(cudaFuncSetAttribute(k_rows_forward_pipe<T, true>, a, bytes));
    upd(cudaFuncSetAttribute(k_rows_inverse_pipe<T, true>, a, bytes));
    upd(cudaFuncSetAttribute(k_theta_forward_pipe<T, true>, a, bytes));
    upd(cudaFuncSetAttribute(k_theta_inverse_pipe<T, true>, a, bytes));
  }
  return e;
}
template <typename T>
cudaError_t pipe_occupancy(int stage, bool adj, int threads, size_t smem, int* bps) {
  constexpr bool fwd_only = std::is_same<T, dd>::value;
  const bool a = adj && !fwd_only;
  switch (stage) {
    case 0: return a ? occupancy_of(k_rows_forward_pipe<T, !fwd_only>, threads, smem, bps)
                     : occupancy_of(k_rows_forward_pipe<T, false>, threads, smem, bps);
    case 1: return a ? occupancy_of(k_theta_forward_pipe<T, !fwd_only>, threads, smem, bps)
                     : occupancy_of(k_theta_forward_pipe<T, false>, threads, smem, bps);
    case 2: return a ? occupancy_of(k_theta_inverse_pipe<T, !fwd_only>, threads, smem, bps)
                     : occupancy_of(k_theta_inverse_pipe<T, false>, threads, smem, bps);
    default: return a ? occupancy_of(k_rows_inverse_pipe<T, !fwd_only>, threads, smem, bps)
                      : occupancy_of(k_rows_inverse_pipe<T, false>, threads, smem, bps);
  }
}

#define SP_INSTANTIATE_PIPE(T)                                                                              \
  template void launch_rows_forward_pipe<T>(bool, const Launch&, const double*, cpx<T>*, int, int, int, int,  \
                                            const FftDesc&, const cpx<T>*, const int*, const cpx<T>*,        \
                                            const double*, const T*, cpx<double>*);                          \
  template void launch_rows_inverse_pipe<T>(bool, const Launch&, const cpx<T>*, double*, int, int, int, int,  \
                                            const FftDesc&, const cpx<T>*, const int*, const cpx<T>*,        \
                                            const double*, const T*, const cpx<double>*);                    \
  template void launch_theta_forward_pipe<T>(bool, const Launch&, cpx<T>*, int, int, int, int, const FftDesc&, \
                                             const cpx<T>*, const int*, const cpx<T>*, T, int);               \
  template void launch_theta_inverse_pipe<T>(bool, const Launch&, cpx<T>*, int, int, int, int, const FftDesc&, \
                                             const cpx<T>*, const int*, const cpx<T>*, T, int);               \
  template cudaError_t pipe_occupancy<T>(int, bool, int, size_t, int*)

}  // namespace sp
