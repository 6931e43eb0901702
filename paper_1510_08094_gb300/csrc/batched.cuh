// Batched solves of many spheres of uneven resolution in one persistent launch.
//
// Every CTA loops: it claims the next problem (problems are ordered largest
// first, so the claim order is a longest-processing-time schedule) from an
// atomic counter, then runs the five stages of that problem itself with its
// own scratch slot for the half spectrum, which stays L2-resident for the
// problem sizes of a batch.  A CTA never waits for another CTA, so the launch
// cannot deadlock whatever the residency.  Problem sizes share per-size
// tables (a BatchClass): twiddles, permutations, factorised eliminations and
// the autotuned transform tiles.
#pragma once

#include "batch_types.h"
#include "kernels.cuh"

namespace sp {

// per-k parity eliminations of one problem by the whole CTA: chain c < K is the
// odd chain of k = c, c >= K the even chain of k = c - K; rows are fetched in
// register batches of U ahead of the dependent recurrence.
__device__ __forceinline__ void solve_chains_cta(cpx<double>* __restrict__ W, const double* __restrict__ fl,
                                                 const double* __restrict__ fiu,
                                                 const double* __restrict__ fcu, int N, int K, int Kp) {
  constexpr int U = 8;
  for (int c = threadIdx.x; c < 2 * K; c += blockDim.x) {
    const bool even = c >= K;
    const int k = even ? c - K : c;
    const int j0 = even ? 2 : 1;
    const double ik2 = k ? 1.0 / ((double)k * (double)k) : 0.0;
    if (j0 >= N) {
      if (even) {
        cpx<double> x0 = W[k];
        W[k] = (k == 0 || (k & 1)) ? cpx<double>{0.0, 0.0} : (-ik2) * x0;
      }
      continue;
    }
    const int M = (N - 1 - j0) / 2 + 1;
    const size_t stride = (size_t)2 * Kp;
    const size_t base = (size_t)j0 * Kp + k;
    cpx<double> y = {0.0, 0.0};
    for (int t0 = 0; t0 < M; t0 += U) {
      cpx<double> d[U];
      double l[U];
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (t0 + q < M) {
          d[q] = W[base + (t0 + q) * stride];
          l[q] = __ldg(fl + base + (t0 + q) * stride);
        }
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (t0 + q < M) {
          y = {fma(-l[q], y.re, d[q].re), fma(-l[q], y.im, d[q].im)};
          W[base + (t0 + q) * stride] = y;
        }
    }
    cpx<double> x = {0.0, 0.0};
    for (int r0 = 0; r0 < M; r0 += U) {
      cpx<double> yv[U];
      double iu[U], cu[U];
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (r0 + q < M) {
          const size_t o = base + (M - 1 - r0 - q) * stride;
          yv[q] = W[o];
          iu[q] = __ldg(fiu + o);
          cu[q] = __ldg(fcu + o);
        }
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (r0 + q < M) {
          x = {fma(yv[q].re, iu[q], -cu[q] * x.re), fma(yv[q].im, iu[q], -cu[q] * x.im)};
          W[base + (M - 1 - r0 - q) * stride] = x;
        }
    }
    if (even && k != 0) {
      // row 0 closure X_0 = (X_2 - F_0)/k^2 (k even), 0 (k odd); k = 0 is closed by theta_inverse
      cpx<double> f0 = W[k];
      if (k & 1) W[k] = {0.0, 0.0};
      else W[k] = {(x.re - f0.re) * ik2, (x.im - f0.im) * ik2};
    }
  }
}

template <bool BIG>
__global__ void __launch_bounds__(256, BIG ? 2 : 3) k_batched_fp64(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* sm = reinterpret_cast<cpx<double>*>(smem_raw);
  __shared__ int s_item;
  cpx<double>* W = a.scratch + (size_t)blockIdx.x * (size_t)a.slot;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.count) break;
    const BatchProblem P = a.problems[a.order[item]];
    const BatchClass& C = a.classes[P.cls];
    const double* f = a.f + P.off;
    double* u = a.u + P.off;
    const double inv_n = 1.0 / (double)C.N;
    const int tr = (C.nt + C.rows - 1) / C.rows;
    const int tc = (C.K + C.cols - 1) / C.cols;
    for (int t = 0; t < tr; ++t) {
      rows_forward_tile<double, false, BIG>(t, sm, f, W, C.nt, C.nl, C.Kp, C.rows, C.row_fft, C.tw_row,
                                            C.perm_row, C.post_row, C.row_scale, C.row_scale, nullptr);
      __syncthreads();
    }
    for (int t = 0; t < tc; ++t) {
      theta_forward_tile<double, false, BIG>(t, sm, W, C.N, C.K, C.Kp, C.cols, C.col_fft, C.tw_col, C.perm_col,
                                             C.post_col_s, inv_n, 1);
      __syncthreads();
    }
    solve_chains_cta(W, C.fl, C.fiu, C.fcu, C.N, C.K, C.Kp);
    __syncthreads();
    for (int t = 0; t < tc; ++t) {
      theta_inverse_tile<double, false, BIG>(t, sm, W, C.N, C.K, C.Kp, C.cols, C.col_fft, C.tw_col, C.perm_col,
                                             C.post_col, inv_n, 1);
      __syncthreads();
    }
    for (int t = 0; t < tr; ++t) {
      rows_inverse_tile<double, false, BIG>(t, sm, W, u, C.nt, C.nl, C.Kp, C.rows, C.row_fft, C.tw_row,
                                            C.perm_row, C.post_row, C.row_scale, C.row_scale, nullptr);
      __syncthreads();
    }
  }
}

}  // namespace sp
