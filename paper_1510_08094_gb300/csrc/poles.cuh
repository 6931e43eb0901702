// Colatitude transforms of the grid with both poles (FP64).
//
// Samples on theta_i = i pi / N, i = 0..N (N + 1 rows: the north pole, the
// interior, the south pole).  Doubled by the glide reflection of eq.
// BMCsphere, the column of wavenumber k lives on theta_p = -pi + 2 pi p / m,
// p = 0..m-1, m = 2N:
//   y_{N+i} = g_i (i = 0..N-1),  y_{N-i} = (-1)^k g_i (i = 1..N; p = 0 is
//   theta = -pi, the south pole), g_i = the longitude transform of row i.
// The pole-free grid folds this doubled column into one DCT-II / DST-II of
// length N; here the doubled samples include theta = 0 and theta = -pi and the
// transform of length m is taken as it stands: one complex FFT of length m per
// column (twice the work of the fold, the same flop count as DCT-I / DST-I of
// length N + 1 on complex data).
//   forward (eq. 2DFourierExpansion):  F_j = (1/m) sum_p y_p exp(-i j theta_p)
//                                          = (-1)^j Y_j / m,  j = 0..N-1,
//     Y the length-m DFT of y;
//   inverse (eq. tildeuFourierExpansion): utilde(theta_p) = sum_{|j| <= N-1}
//     X_j exp(i j theta_p) with X_{-j} = (-1)^k X_j (the BMC symmetry) and the
//     theta-Nyquist mode dropped: the inverse DFT of z, z_j = (-1)^j X_j,
//     z_{m-j} = (-1)^{j+k} X_j (j = 1..N-1), z_N = 0; row i <- p = N + i
//     (i < N), row N <- p = 0 (theta = -pi is theta = pi).
// The CTA of k = 0 closes the zero-mean row first (zonal_closure, as the
// pole-free inverse does).  One column per CTA, the length-m column in shared memory (digit-reversed
// load, decimation in time, as fft_run).  The spectrum array W holds N + 1
// rows: the forward reads rows 0..N of column k and writes rows 0..N-1, the
// inverse reads rows 0..N-1 and writes rows 0..N.
#pragma once

#include "kernels.cuh"

namespace sp {

template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_forward_poles(
    cpx<double>* __restrict__ W, int N, int K, int Kp, FftDesc d, const cpx<double>* __restrict__ tw,
    const int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* sm = reinterpret_cast<cpx<double>*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= K) return;                       // uniform over the block
  const int m = 2 * N;
  const bool odd = (k & 1) != 0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    const int i = p >= N ? p - N : N - p;   // the sample row of theta_p
    cpx<double> v = W[(size_t)i * Kp + k];
    if (p < N && odd) v = {-v.re, -v.im};
    sm[__ldg(perm + p)] = v;
  }
  __syncthreads();
  fft_run<-1, BIG>(sm, 1, d, tw);
  __syncthreads();
  const double inv_m = 1.0 / (double)m;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const cpx<double> y = sm[j];
    const double s = (j & 1) ? -inv_m : inv_m;
    W[(size_t)j * Kp + k] = {y.re * s, y.im * s};
  }
}

template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_inverse_poles(
    cpx<double>* __restrict__ W, int N, int K, int Kp, FftDesc d, const cpx<double>* __restrict__ tw,
    const int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* sm = reinterpret_cast<cpx<double>*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= K) return;
  // k = 0: the solve leaves the zero-mean closure w^T X_0 = 0 to the inverse
  // transform, X_00 = sum_{j even >= 2} 2 X_j0/(j^2-1), as on the pole-free grid
  if (k == 0) zonal_closure(W, N, Kp);
  const int m = 2 * N;
  const bool odd = (k & 1) != 0;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    cpx<double> v = {0.0, 0.0};
    if (q < N) {
      v = W[(size_t)q * Kp + k];
      if (q & 1) v = {-v.re, -v.im};
    } else if (q > N) {
      const int j = m - q;
      v = W[(size_t)j * Kp + k];
      if (((j & 1) != 0) != odd) v = {-v.re, -v.im};
    }
    sm[__ldg(perm + q)] = v;
  }
  __syncthreads();
  fft_run<+1, BIG>(sm, 1, d, tw);
  __syncthreads();
  for (int i = threadIdx.x; i <= N; i += blockDim.x) W[(size_t)i * Kp + k] = sm[i < N ? N + i : 0];
}

// ---------------------------------------------------------------------------
// The adjoint (ubar -> fbar) runs the conjugate transposes of the two maps
// above, per column, with the same FFT:
//   of the inverse (first colatitude stage of the adjoint): with G_p = Ubar at
//     the rows' positions (p = N + i for row i < N, p = 0 for row N, zero at
//     p = 1..N-1) and Y its length-m DFT (exp(-2 pi i q p / m)),
//       Xbar_0 = Y_0,  Xbar_j = (-1)^j (Y_j + (-1)^k Y_{m-j}),  j = 1..N-1,
//     and for k = 0 the transpose of the zero-mean closure:
//       Xbar_j += 2 Xbar_0 / (j^2 - 1) for even j >= 2;
//   of the forward (last colatitude stage of the adjoint): with v the inverse
//     DFT of z_q = (-1)^q Fbar_q (q < N, zero above),
//       gbar_i = (v_{N+i} [i < N] + (-1)^k v_{N-i} [i >= 1]) / m,  i = 0..N.
// ---------------------------------------------------------------------------
template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_poles_adj_first(
    cpx<double>* __restrict__ W, int N, int K, int Kp, FftDesc d, const cpx<double>* __restrict__ tw,
    const int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* sm = reinterpret_cast<cpx<double>*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= K) return;
  const int m = 2 * N;
  const bool odd = (k & 1) != 0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    cpx<double> v = {0.0, 0.0};
    if (p >= N) v = W[(size_t)(p - N) * Kp + k];
    else if (p == 0) v = W[(size_t)N * Kp + k];
    sm[__ldg(perm + p)] = v;
  }
  __syncthreads();
  fft_run<-1, BIG>(sm, 1, d, tw);
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    cpx<double> y = sm[j];
    if (j > 0) {
      const cpx<double> yc = sm[m - j];
      y = odd ? cpx<double>{y.re - yc.re, y.im - yc.im} : cpx<double>{y.re + yc.re, y.im + yc.im};
    }
    if (j & 1) y = {-y.re, -y.im};
    W[(size_t)j * Kp + k] = y;
  }
  if (k == 0) {     // uniform over the block
    __syncthreads();
    const cpx<double> x0 = W[0];
    for (int j = 2 + 2 * (int)threadIdx.x; j < N; j += 2 * (int)blockDim.x) {
      const double w = 2.0 / ((double)j * (double)j - 1.0);
      cpx<double>& x = W[(size_t)j * Kp];
      x = {fma(w, x0.re, x.re), fma(w, x0.im, x.im)};
    }
  }
}

template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_poles_adj_last(
    cpx<double>* __restrict__ W, int N, int K, int Kp, FftDesc d, const cpx<double>* __restrict__ tw,
    const int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* sm = reinterpret_cast<cpx<double>*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= K) return;
  const int m = 2 * N;
  const bool odd = (k & 1) != 0;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    cpx<double> v = {0.0, 0.0};
    if (q < N) {
      v = W[(size_t)q * Kp + k];
      if (q & 1) v = {-v.re, -v.im};
    }
    sm[__ldg(perm + q)] = v;
  }
  __syncthreads();
  fft_run<+1, BIG>(sm, 1, d, tw);
  __syncthreads();
  const double inv_m = 1.0 / (double)m;
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
    cpx<double> g = {0.0, 0.0};
    if (i < N) g = sm[N + i];
    if (i >= 1) {
      const cpx<double> t = sm[N - i];
      g = odd ? cpx<double>{g.re - t.re, g.im - t.im} : cpx<double>{g.re + t.re, g.im + t.im};
    }
    W[(size_t)i * Kp + k] = {g.re * inv_m, g.im * inv_m};
  }
}

}  // namespace sp
