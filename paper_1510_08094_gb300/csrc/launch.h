// Host-side launchers of the transform and elimination kernels.  Each
// arithmetic type's kernels are compiled in their own translation unit
// (k_f64.cu, k_f32.cu, k_dd.cu); the plan code in sphere_poisson.cu only sees
// these declarations.
#pragma once

#include <cuda_runtime.h>

#include "batch_types.h"
#include "fft.cuh"

namespace sp {

struct Launch {
  dim3 grid;
  int threads;
  size_t smem;
  cudaStream_t stream;
};

template <typename T>
void launch_rows_forward(bool adj, bool big, const Launch& l, const double* f, cpx<T>* W, int nt, int n,
                         int Kp, int rows, const FftDesc& d, const cpx<T>* tw, const int* perm,
                         const cpx<T>* post, const double* row_scale, const T* row_scale_t,
                         cpx<double>* zonal);
template <typename T>
void launch_rows_inverse(bool adj, bool big, const Launch& l, const cpx<T>* W, double* u, int nt, int n,
                         int Kp, int rows, const FftDesc& d, const cpx<T>* tw, const int* perm,
                         const cpx<T>* post, const double* row_scale, const T* row_scale_t,
                         const cpx<double>* zonal);
template <typename T>
void launch_theta_forward(bool adj, bool big, const Launch& l, cpx<T>* W, int N, int K, int Kp, int cols,
                          const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                          int zonal);
template <typename T>
void launch_theta_inverse(bool adj, bool big, const Launch& l, cpx<T>* W, int N, int K, int Kp, int cols,
                          const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                          int zonal);
// Pipelined (persistent) forms of the four transform kernels: grid = a
// number of resident CTAs, each looping over tiles while cp.async stages its
// next tile's input; dynamic shared memory = the FFT buffer plus the staged
// input (16-byte aligned after it).  Non-BIG radices only.
template <typename T>
void launch_rows_forward_pipe(bool adj, const Launch& l, const double* f, cpx<T>* W, int nt, int n, int Kp,
                              int rows, const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post,
                              const double* row_scale, const T* row_scale_t, cpx<double>* zonal);
template <typename T>
void launch_rows_inverse_pipe(bool adj, const Launch& l, const cpx<T>* W, double* u, int nt, int n, int Kp,
                              int rows, const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post,
                              const double* row_scale, const T* row_scale_t, const cpx<double>* zonal);
template <typename T>
void launch_theta_forward_pipe(bool adj, const Launch& l, cpx<T>* W, int N, int K, int Kp, int cols,
                               const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                               int zonal);
template <typename T>
void launch_theta_inverse_pipe(bool adj, const Launch& l, cpx<T>* W, int N, int K, int Kp, int cols,
                               const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                               int zonal);
// CTAs per SM of pipelined kernel `stage` (0 rows_forward, 1 theta_forward,
// 2 theta_inverse, 3 rows_inverse); sets its shared-memory cap to `smem`
template <typename T>
cudaError_t pipe_occupancy(int stage, bool adj, int threads, size_t smem, int* blocks_per_sm);

// raise the dynamic shared-memory cap of T's transform kernels
template <typename T>
cudaError_t allow_transform_smem(int bytes);

template <typename S>
void launch_solve(bool adj, const Launch& l, cpx<S>* W, const S* fl, const S* fiu, const S* fcu, int N, int K,
                  int Kp);
// twist: the twisted factorisation k_solve and k_refine need; false: the
// top-down one of the zonal scan and the batched kernels
template <typename S>
void launch_factor(const Launch& l, S* fl, S* fiu, S* fcu, int N, int K, int Kp, bool twist);

// the FP32 form's fused colatitude stage (forward transform, parity
// eliminations, inverse transform per column tile; fused.cuh): tables of
// launch_factor_cols, one CTA per tile of `cols` columns with a transform
// buffer and a coefficient buffer; cols < 0: -cols columns per CTA in one
// buffer (decimation-in-frequency inverse); cols = 0: one column per CTA in
// clusters of four that share their loads and stores (l.grid is ignored);
// theta_fused_smem dynamic bytes
// The single-buffer form with two columns per CTA takes its tile by TMA when a
// tensor map of W can be encoded and `status` (a device int) is given; status
// receives kStatusTmaTimeout if the bounded wait gives up.
void launch_theta_fused(bool big, const Launch& l, cpx<float>* W, int N, int K, int Kp, int cols, const FftDesc& d,
                        const cpx<float>* tw, const int* perm, const cpx<float>* post_s, const cpx<float>* post,
                        const float* fiu, float inv_n, int* status);
size_t theta_fused_smem(int N, int cols, int threads);
// the adjoint's colatitude stage (transposed transforms and eliminations) in
// one launch: the single-buffer form, -cols columns per CTA (cols < 0; 1 else),
// theta_fused_smem(N, cols, threads) bytes, post the unscaled DCT table
void launch_theta_fused_adj(bool big, const Launch& l, cpx<float>* W, int N, int K, int Kp, int cols,
                            const FftDesc& d, const cpx<float>* tw, const int* perm, const cpx<float>* post,
                            const float* fiu, float inv_n, int* status);
// the colatitude transforms of the grid with both poles (poles.cuh): one CTA
// per column k < K (grid K), 2N complex doubles of dynamic shared memory;
// d, tw and perm describe the length-2N FFT
void launch_theta_poles(bool inverse, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                        const FftDesc& d, const cpx<double>* tw, const int* perm);
// their conjugate transposes for the adjoint: last = false the transpose of the
// inverse (the adjoint's first colatitude stage, with the zero-mean closure's
// transpose), last = true the transpose of the forward
void launch_theta_poles_adj(bool last, bool big, const Launch& l, cpx<double>* W, int N, int K, int Kp,
                            const FftDesc& d, const cpx<double>* tw, const int* perm);
// the FP32 + refinement form's fused colatitude stage (fused_refine.cuh): one
// CTA per column k >= 1 (column 0 is the FP64 zonal path's), in place in W
// (double-float spectrum); refine_fused_smem dynamic bytes
// The next columns' samples are copied by the tensor memory accelerator when
// a tensor map of W can be encoded and `status` (a device int) is given, else
// by cp.async; status receives kStatusTmaTimeout if a TMA wait gives up.
void launch_refine_fused(bool big, const Launch& l, cpx<dd>* W, int N, int K, int Kp, const FftDesc& d,
                         const cpx<dd>* tw, const int* perm, const cpx<dd>* post_s, const cpx<dd>* post,
                         const float* fiu, int sweeps, int* status);
size_t refine_fused_smem(int N, int threads);
// a bounded wait that runs out: sets *status (device) to kStatusTmaTimeout
void launch_wait_selftest(int* status, unsigned polls, cudaStream_t st);
// pivots 1/u of the top-down factorisation of every parity chain, stored per
// column ([k][j]), 2K threads
void launch_factor_cols(const Launch& l, float* fiu, int N, int K);

// FP64 zonal-column eliminations by parallel scan (one CTA)
void launch_zonal_scan(bool adj, cudaStream_t st, cpx<double>* Z, const double* zl, const double* ziu,
                       const double* zcu, int N);

// persistent batched FP64 solve: set the kernel's shared-memory cap and report
// how many CTAs of `threads` fit per SM with `smem` dynamic bytes
cudaError_t batched_fp64_occupancy(bool big, int threads, size_t smem, int* blocks_per_sm);
void launch_batched_fp64(bool big, dim3 grid, int threads, size_t smem, cudaStream_t st, const BatchArgs& a);
// the same for the persistent batched FP32 + refinement solve
cudaError_t batched_refine_occupancy(bool big, int threads, size_t smem, int* blocks_per_sm);
void launch_batched_refine(bool big, dim3 grid, int threads, size_t smem, cudaStream_t st, const BatchArgs& a);

// surface integral from the k = 0 coefficient column (one CTA, result to device memory)
void launch_sum2_finish(cudaStream_t st, const cpx<double>* C, int N, int Kp, double* out);
// mean of f over the sphere and max |f| (either output may be NULL): `nparts`
// partial sums in part[0..nparts) (device scratch), then one CTA adds them
void launch_mean(cudaStream_t st, const double* f, int nt, int n, const double* wrow, double2* part, int nparts,
                 double* mean, double* absmax);
// tangential derivatives: Q = (1/sin theta) d/dlambda in coefficients (the
// scratch array P of msin_scratch_bytes bytes takes the chunk sums), then the
// signed sums of gradient components that `tc` describes
size_t msin_scratch_bytes(int N, int Kp);
void launch_msin_div(cudaStream_t st, const cpx<double>* X, cpx<double>* Q, cpx<double>* P, int N, int K, int Kp);
void launch_tangential(cudaStream_t st, const cpx<double>* X, const cpx<double>* Q, const TangentialCombo& tc,
                       int N, int K, int Kp);
// X_jk = 0 where |X_jk| <= rtol max |X| (mx: one device word of scratch)
void launch_coeff_chop(cudaStream_t st, cpx<double>* X, int N, int K, int Kp, unsigned long long* mx,
                       double rtol);
// pointwise with the unit normal on the grid (geo: sin, cos theta; cos, sin lambda):
// (a, b, c) <- n x (a, b, c), and out = n . (a, b, c) (out may be c)
void launch_cross_normal(cudaStream_t st, double* a, double* b, double* c, const double* geo, int nt, int nl);
void launch_normal_dot(cudaStream_t st, const double* a, const double* b, const double* c, double* out,
                       const double* geo, int nt, int nl);

// structure-preserving GE: pivot search (partials + final into *out) and one
// step (extract the term's column and row, update the residual; AB: 2 n
// doubles of scratch)
void launch_ge_pivot(cudaStream_t st, const double* e, int nt, int n, GePivot* part, int nparts, GePivot* out);
void launch_ge_step(cudaStream_t st, double* e, int nt, int n, int istar, int qstar, double* col, double* row,
                    double p0, double p1, double* AB);
// low-rank right-hand side: pack the terms' columns for theta_forward, then F
void launch_lowrank_pack(cudaStream_t st, const double* cols, int terms, int nt, const double* sin2, cpx<double>* Wc);
// (scales Wc in place by the pivot weights first)
void launch_lowrank_outer(cudaStream_t st, cpx<double>* Wc, const cpx<double>* R, const double* piv,
                          int terms, int N, int K, int Kp, cpx<double>* F);

void launch_refine(const Launch& l, const cpx<dd>* F, cpx<dd>* X, cpx<float>* Y, const float* fl,
                   const float* fiu, const float* fcu, int N, int K, int Kp, int first);
void launch_zonal_extract(const Launch& l, const cpx<dd>* Wdd, cpx<double>* Z, int N, int Kp);
void launch_zonal_insert(const Launch& l, const cpx<double>* Z, cpx<dd>* X, int N, int Kp);

}  // namespace sp
