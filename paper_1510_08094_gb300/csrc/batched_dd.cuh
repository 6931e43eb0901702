// Batched FP32 + refinement solves: many spheres of uneven resolution in one
// persistent launch, in the arithmetic of the single-plan SP_FP32_REFINE form.
//
// Per problem the claiming CTA runs: the double-float longitude and colatitude
// transforms (F in double-float, Section 5's 2D Fourier coefficients of
// sin^2(theta) f), the eliminations of eq. linearSystems for k >= 1 as FP32
// Thomas sweeps on the parity tridiagonals refined by double-float residuals
// R = F - L X, the k = 0 column (the ill-conditioned zonal system with the
// w^T X_0 = 0 row of eq. pentdiagonalPlusRankOne) in FP64, and the inverse
// double-float transforms.  The work queue, the scratch slot per CTA and the
// size-class tables are those of the FP64 batched kernel.
#pragma once

#include "batch_types.h"
#include "kernels.cuh"

namespace sp {

// All sweeps of one chain (k >= 1, j = j0, j0 + 2, ... < N) by one thread.
//   sweep s: R_t = F_t - (a_t X_{t-1} + b_t X_t + c_t X_{t+1})  (s = 0: R = F, X = 0)
//            y_t = R_t - l_t y_{t-1}            (FP32, y kept in Y)
//            d_t = y_t/u_t - (c_t/u_t) d_{t+1}  (FP32)
//            X_t += d_t                         (double-float)
// a_t = (j-1)(j-2)/4, b_t = -(j^2 + 2k^2)/2, c_t = (j+1)(j+2)/4, formed exactly
// from FP32 products of integers.  Rows are fetched in register batches of U
// ahead of the dependent recurrences.
__device__ __forceinline__ void refine_chain(const cpx<dd>* __restrict__ F, cpx<dd>* __restrict__ X,
                                             cpx<float>* __restrict__ Y, const float* __restrict__ fl,
                                             const float* __restrict__ fiu, const float* __restrict__ fcu,
                                             int N, int Kp, int k, bool even, int sweeps) {
  constexpr int U = 4;
  const int j0 = even ? 2 : 1;
  const cpx<dd> zero = {dd(0.f, 0.f), dd(0.f, 0.f)};
  if (j0 < N) {
    const int M = (N - 1 - j0) / 2 + 1;
    const size_t stride = (size_t)2 * Kp;
    const size_t base = (size_t)j0 * Kp + k;
    const float kf = (float)k;
    const dd two_k2 = dd_mul(dd_prod(kf, kf), dd(2.f, 0.f));
    for (int s = 0; s <= sweeps; ++s) {
      const bool first = s == 0;
      cpx<dd> xm1 = zero, x0 = first ? zero : X[base];
      cpx<float> y = {0.f, 0.f};
      float jf = (float)j0;
      for (int t0 = 0; t0 < M; t0 += U) {
        cpx<dd> fv[U], xv[U];
        float lv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          const int t = t0 + q;
          xv[q] = zero;
          if (t < M) {
            fv[q] = F[base + t * stride];
            lv[q] = __ldg(fl + base + t * stride);
            if (!first && t + 1 < M) xv[q] = X[base + (t + 1) * stride];
          }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
          if (t0 + q < M) {
            cpx<dd> r = fv[q];
            if (!first) {
              dd a = dd_prod(jf - 1.f, jf - 2.f);
              a = dd(a.hi * 0.25f, a.lo * 0.25f);
              dd b = dd_add(dd_prod(jf, jf), two_k2);
              b = dd(b.hi * -0.5f, b.lo * -0.5f);
              dd c = dd_prod(jf + 1.f, jf + 2.f);
              c = dd(c.hi * 0.25f, c.lo * 0.25f);
              cpx<dd> lx = cdd_scale(b, x0);
              lx = {dd_fma(a, xm1.re, lx.re), dd_fma(a, xm1.im, lx.im)};
              lx = {dd_fma(c, xv[q].re, lx.re), dd_fma(c, xv[q].im, lx.im)};
              r = {dd_sub(r.re, lx.re), dd_sub(r.im, lx.im)};
            }
            const cpx<float> rf = {r.re.hi + r.re.lo, r.im.hi + r.im.lo};
            y = {fmaf(-lv[q], y.re, rf.re), fmaf(-lv[q], y.im, rf.im)};
            Y[base + (t0 + q) * stride] = y;
            xm1 = x0;
            x0 = xv[q];
            jf += 2.f;
          }
        }
      }
      cpx<float> dl = {0.f, 0.f};
      for (int r0 = 0; r0 < M; r0 += U) {
        cpx<float> yv[U];
        cpx<dd> xv[U];
        float iu[U], cu[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          xv[q] = zero;
          if (r0 + q < M) {
            const size_t o = base + (size_t)(M - 1 - r0 - q) * stride;
            yv[q] = Y[o];
            iu[q] = __ldg(fiu + o);
            cu[q] = __ldg(fcu + o);
            if (!first) xv[q] = X[o];
          }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
          if (r0 + q < M) {
            dl = {fmaf(yv[q].re, iu[q], -cu[q] * dl.re), fmaf(yv[q].im, iu[q], -cu[q] * dl.im)};
            const cpx<dd> x = {dd_add(xv[q].re, dd(dl.re, 0.f)), dd_add(xv[q].im, dd(dl.im, 0.f))};
            X[base + (size_t)(M - 1 - r0 - q) * stride] = x;
          }
        }
      }
    }
  }
  if (even) {
    // row 0: X_0 = (X_2 - F_0)/k^2 for k even (X_{-2,k} = X_{2,k}), 0 for k odd
    cpx<dd> x0v = zero;
    if (!(k & 1)) {
      const cpx<dd> x2 = (2 < N) ? X[(size_t)2 * Kp + k] : zero;
      const cpx<dd> f0 = F[k];
      const dd ik2 = dd_from_double(1.0 / ((double)k * (double)k));
      x0v = {dd_mul(dd_sub(x2.re, f0.re), ik2), dd_mul(dd_sub(x2.im, f0.im), ik2)};
    }
    X[k] = x0v;
  }
}

// One k = 0 chain in FP64 with the plan's FP64 factors (zl, ziu, zcu at
// [j][0] of an [N][2] table).  The FP64 values are parked in X's column-0
// slots (a complex double-float and a complex double are both 16 bytes) until
// zonal_finish converts them.
__device__ __forceinline__ void zonal_chain(const cpx<dd>* __restrict__ F, cpx<dd>* __restrict__ X,
                                            const double* __restrict__ zl, const double* __restrict__ ziu,
                                            const double* __restrict__ zcu, int N, int Kp, bool even) {
  constexpr int U = 4;
  const int j0 = even ? 2 : 1;
  if (j0 >= N) return;
  const int M = (N - 1 - j0) / 2 + 1;
  static_assert(sizeof(cpx<dd>) == sizeof(cpx<double>), "parked FP64 values share the slots");
  cpx<double>* Xd = reinterpret_cast<cpx<double>*>(X);
  auto xslot = [&](int j) -> cpx<double>& { return Xd[(size_t)j * Kp]; };
  cpx<double> y = {0.0, 0.0};
  for (int t0 = 0; t0 < M; t0 += U) {
    cpx<double> d[U];
    double l[U];
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (t0 + q < M) {
        const int j = j0 + 2 * (t0 + q);
        const cpx<dd> fv = F[(size_t)j * Kp];
        d[q] = {dd_to_double(fv.re), dd_to_double(fv.im)};
        l[q] = __ldg(zl + 2 * (size_t)j);
      }
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (t0 + q < M) {
        y = {fma(-l[q], y.re, d[q].re), fma(-l[q], y.im, d[q].im)};
        xslot(j0 + 2 * (t0 + q)) = y;
      }
  }
  cpx<double> x = {0.0, 0.0};
  for (int r0 = 0; r0 < M; r0 += U) {
    cpx<double> yv[U];
    double iu[U], cu[U];
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (r0 + q < M) {
        const int j = j0 + 2 * (M - 1 - r0 - q);
        yv[q] = xslot(j);
        iu[q] = __ldg(ziu + 2 * (size_t)j);
        cu[q] = __ldg(zcu + 2 * (size_t)j);
      }
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (r0 + q < M) {
        x = {fma(yv[q].re, iu[q], -cu[q] * x.re), fma(yv[q].im, iu[q], -cu[q] * x.im)};
        xslot(j0 + 2 * (M - 1 - r0 - q)) = x;
      }
  }
}

// Close the zonal column with w^T X_0 = 0, X_00 = sum_{j even >= 2} 2 X_j0/(j^2-1)
// (X_{-j,0} = X_{j,0}), and convert column 0 from the parked FP64 values to
// double-float.  Whole CTA; `red` holds one value per warp.
__device__ __forceinline__ void zonal_finish(cpx<dd>* __restrict__ X, int N, int Kp, cpx<double>* red) {
  cpx<double>* Xd = reinterpret_cast<cpx<double>*>(X);
  cpx<double> acc = {0.0, 0.0};
  for (int j = 2 + 2 * threadIdx.x; j < N; j += 2 * blockDim.x) {
    const double wj = 2.0 / ((double)j * (double)j - 1.0);
    acc = acc + wj * Xd[(size_t)j * Kp];
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc.re = acc.re + __shfl_down_sync(0xffffffffu, acc.re, off);
    acc.im = acc.im + __shfl_down_sync(0xffffffffu, acc.im, off);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  for (int j = 1 + threadIdx.x; j < N; j += blockDim.x) {
    const cpx<double> v = Xd[(size_t)j * Kp];
    X[(size_t)j * Kp] = {dd_from_double(v.re), dd_from_double(v.im)};
  }
  if (threadIdx.x == 0) {
    cpx<double> tot = {0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot = tot + red[w];
    X[0] = {dd_from_double(tot.re), dd_from_double(tot.im)};
  }
}

// Scratch slot of a CTA for a problem of class C: F and X (complex double-float,
// N x Kp each, 16 bytes an element) then Y (complex FP32, N x Kp): 40 bytes per
// spectral element.
template <bool BIG>
__global__ void __launch_bounds__(256, 2) k_batched_refine(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<dd>* sm = reinterpret_cast<cpx<dd>*>(smem_raw);
  __shared__ int s_item;
  __shared__ cpx<double> red[32];
  cpx<double>* slot = a.scratch + (size_t)blockIdx.x * (size_t)a.slot;
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
    const size_t nkp = (size_t)C.N * C.Kp;
    cpx<dd>* F = reinterpret_cast<cpx<dd>*>(slot);
    cpx<dd>* X = F + nkp;
    cpx<float>* Y = reinterpret_cast<cpx<float>*>(X + nkp);
    const dd inv_n = dd_from_double(1.0 / (double)C.N);
    const int tr = (C.nt + C.rows - 1) / C.rows;
    const int tc = (C.K + C.cols - 1) / C.cols;
    for (int t = 0; t < tr; ++t) {
      rows_forward_tile<dd, false, BIG>(t, sm, f, F, C.nt, C.nl, C.Kp, C.rows, C.row_fft, C.tw_row_d,
                                        C.perm_row, C.post_row_d, C.row_scale, C.row_scale_d, nullptr);
      __syncthreads();
    }
    for (int t = 0; t < tc; ++t) {
      theta_forward_tile<dd, false, BIG>(t, sm, F, C.N, C.K, C.Kp, C.cols, C.col_fft, C.tw_col_d, C.perm_col,
                                         C.post_col_s_d, inv_n, 0);
      __syncthreads();
    }
    // chain c < K: odd chain of k = c; c >= K: even chain of k = c - K; k = 0 in FP64
    for (int c = threadIdx.x; c < 2 * C.K; c += blockDim.x) {
      const bool even = c >= C.K;
      const int k = even ? c - C.K : c;
      if (k == 0) zonal_chain(F, X, C.zl, C.ziu, C.zcu, C.N, C.Kp, even);
      else refine_chain(F, X, Y, C.fl32, C.fiu32, C.fcu32, C.N, C.Kp, k, even, a.sweeps);
    }
    __syncthreads();
    zonal_finish(X, C.N, C.Kp, red);
    __syncthreads();
    for (int t = 0; t < tc; ++t) {
      theta_inverse_tile<dd, false, BIG>(t, sm, X, C.N, C.K, C.Kp, C.cols, C.col_fft, C.tw_col_d, C.perm_col,
                                         C.post_col_d, inv_n, 0);
      __syncthreads();
    }
    for (int t = 0; t < tr; ++t) {
      rows_inverse_tile<dd, false, BIG>(t, sm, X, u, C.nt, C.nl, C.Kp, C.rows, C.row_fft, C.tw_row_d,
                                        C.perm_row, C.post_row_d, C.row_scale, C.row_scale_d, nullptr);
      __syncthreads();
    }
  }
}

}  // namespace sp
