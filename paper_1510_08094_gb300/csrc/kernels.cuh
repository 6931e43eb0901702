// Device kernels of the spherical Poisson solve (Section 5), one per stage.
//
// Data flow of one solve (n = n_lambda, L = n/2, N = n_theta, K = L + 1
// half-spectrum wavenumbers, Kp = K rounded up to even, workspace W[N][Kp]):
//   rows_forward   f[N][n]  -> W: G_i(k) = sin^2(theta_i)/n * sum_q f_iq e^{-2 pi i k q/n}
//                  (real FFT of each colatitude row through a length-L complex FFT)
//   theta_forward  W -> W:  per k, the length-2N DFS transform of the column,
//                  folded by the BMC symmetry X_{-j,k} = (-1)^k X_{j,k}: a DCT-II
//                  (k even) or DST-II (k odd) of length N, each through one
//                  length-N complex FFT (Makhoul's reordering), scaled 1/N
//   solve          W -> W:  per k, rows j >= 1 split by parity into two
//                  tridiagonal systems (offsets 0, +-2 of eq. linearSystems),
//                  eliminated with factors precomputed at plan time; then the
//                  j = 0 closure (row 0 for k != 0, w^T X_0 = 0 for k = 0)
//   theta_inverse  W -> W:  DCT-III / DST-III back to colatitude samples
//   rows_inverse   W -> u[N][n]: inverse real FFT of each row
// The adjoint runs the transposed stages in reverse order (ADJ = true); each
// transposed stage is the other transform family with different weights.
#pragma once

#include <type_traits>

#include "batch_types.h"
#include "fft.cuh"

namespace sp {

// position of colatitude sample i in Makhoul's reordering: even samples first,
// odd samples reversed at the end (v_p = x_{2p}, v_{N-1-p} = x_{2p+1})
__device__ __forceinline__ int makhoul_pos(int i, int N) {
  return (i & 1) ? N - 1 - (i >> 1) : (i >> 1);
}

// cp.async: asynchronous global -> shared copies (16 bytes through L2, 8 through L1)
__device__ __forceinline__ void cp_async16(void* smem, const void* g) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* g) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Split of a double into two floats hi + lo (|x - hi - lo| <= 2^-48 |x|) with
// integer operations only: hi keeps the top 24 significand bits (truncated),
// lo the next 29 bits rounded to 24.  Used where FP64-accurate sums of double
// inputs are needed without spending the scarce FP64 pipe.  Values outside the
// float range (and subnormals) give 0 / infinity.
__device__ __forceinline__ dd split_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7ffu);
  const int fe = e - 1023 + 127;
  if (e == 0 || fe <= 0) return dd(0.f, 0.f);
  if (e == 0x7ff || fe >= 255) return dd(__uint_as_float(sign | 0x7f800000u | ((e == 0x7ff && ((h32 & 0xfffffu) | l32)) ? 0x400000u : 0u)), 0.f);
  const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | m23);
  const int se = e - 1075 + 127;                 // exponent of the unit of the low 29 bits
  float lo = 0.f;
  if (se > 0) lo = __fmul_rn(__uint2float_rn(l32 & 0x1fffffffu), __uint_as_float((unsigned)se << 23));
  return dd(hi, sign ? -lo : lo);
}

// Exact float -> double with integer operations only (a float is exactly a
// double): rebias the exponent and widen the significand.  Subnormal floats
// are taken as zero; infinities and NaNs are kept.
__device__ __forceinline__ double float_to_double_int(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned m = b & 0x7fffffu;
  unsigned hi;
  if (e == 0) hi = sign;                                       // zero (and subnormals)
  else if (e == 0xffu) hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
  else hi = sign | ((e + 896u) << 20) | (m >> 3);
  const unsigned lo = m << 29;
  return __hiloint2double((int)hi, (int)(e == 0 ? 0u : lo));
}

// double -> float without the FP64 pipe: hi + lo of the integer split, rounded once
__device__ __forceinline__ float double_to_float_int(double x);

__device__ __forceinline__ dd warp_sum_dd(dd v) {
  for (int off = 16; off > 0; off >>= 1) {
    dd o(__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off));
    v = dd_add(v, o);
  }
  return v;
}

// block-wide double-float sum (result valid in thread 0); all threads must call
__device__ __forceinline__ float double_to_float_int(double x) {
  dd s = split_double(x);
  return __fadd_rn(s.hi, s.lo);
}

// input conversion of the transforms: double -> T without the FP64 pipe
template <typename T> __device__ __forceinline__ T load_conv(double x);
template <> __device__ __forceinline__ double load_conv<double>(double x) { return x; }
template <> __device__ __forceinline__ float load_conv<float>(double x) { return double_to_float_int(x); }
template <> __device__ __forceinline__ dd load_conv<dd>(double x) {
  dd s = split_double(x);
  float h = __fadd_rn(s.hi, s.lo);                 // renormalise the split
  return dd(h, __fsub_rn(s.lo, __fsub_rn(h, s.hi)));
}
// output conversion T -> double (float: integer widening; double-float: two
// widenings and one FP64 add)
template <typename T> __device__ __forceinline__ double store_conv(T x);
template <> __device__ __forceinline__ double store_conv<double>(double x) { return x; }
template <> __device__ __forceinline__ double store_conv<float>(float x) { return float_to_double_int(x); }
template <> __device__ __forceinline__ double store_conv<dd>(dd x) {
  return float_to_double_int(x.hi) + float_to_double_int(x.lo);
}

__device__ __forceinline__ dd block_sum_dd(dd v) {
  __shared__ dd red_dd[32];
  v = warp_sum_dd(v);
  if ((threadIdx.x & 31) == 0) red_dd[threadIdx.x >> 5] = v;
  __syncthreads();
  dd t(0.f, 0.f);
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = dd_add(t, red_dd[w]);
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// Tile inputs.  Every transform kernel first gathers its tile into the FFT
// buffer (permuted, pre-processed); the input is read either straight from
// global memory or from a copy of the tile that cp.async staged in shared
// memory while the previous tile was being transformed (the pipelined
// kernels below).  Element (r, q): row r of the tile, entry q of that row.
// ---------------------------------------------------------------------------
template <typename E>
struct FromGlobal {
  const E* p;    // element (0, 0)
  size_t ld;     // row stride in elements
  __device__ __forceinline__ E operator()(int r, int q) const { return p[(size_t)r * ld + q]; }
};
template <typename E>
struct FromStaged {
  const E* p;    // shared memory
  int ld;
  __device__ __forceinline__ E operator()(int r, int q) const { return p[r * ld + q]; }
};
// read-only double pairs of f (rows_forward from global memory)
struct FromInput {
  const double2* p;
  size_t ld;
  __device__ __forceinline__ double2 operator()(int r, int q) const { return __ldg(p + (size_t)r * ld + q); }
};

// cp.async copies of `rows` rows of `bytes` bytes each (a multiple of CH = 16
// or 8) from g (row stride ld_bytes) to consecutive rows of S.
template <int CH>
__device__ __forceinline__ void cp_async_chunk(void* s, const void* g) {
  if constexpr (CH == 16) cp_async16(s, g);
  else cp_async8(s, g);
}
template <int CH>
__device__ __forceinline__ void stage_rows(void* S, const void* g, size_t ld_bytes, int rows, int bytes) {
  const int per = bytes / CH;
  for (int r = 0; r < rows; ++r) {
    const char* src = static_cast<const char*>(g) + (size_t)r * ld_bytes;
    char* dst = static_cast<char*>(S) + (size_t)r * bytes;
    for (int c = threadIdx.x; c < per; c += blockDim.x) cp_async_chunk<CH>(dst + c * CH, src + c * CH);
  }
}
// the same for many short rows (the colatitude tiles: N rows of `cols`
// elements): `valid` chunks of each row are copied, the thread loop runs over
// 1 << ps >= valid chunk slots per row
template <int CH>
__device__ __forceinline__ void stage_columns(void* S, const void* g, size_t ld_bytes, int nrows, int ps,
                                              int valid, int row_bytes) {
  const int total = nrows << ps;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int r = t >> ps, c = t & ((1 << ps) - 1);
    if (c < valid)
      cp_async_chunk<CH>(static_cast<char*>(S) + (size_t)r * row_bytes + c * CH,
                         static_cast<const char*>(g) + (size_t)r * ld_bytes + c * CH);
  }
}

// ---------------------------------------------------------------------------
// rows_forward: real FFT along longitude in arithmetic T.
//   forward (ADJ = false): W[i][k] = row_scale[i] * G_i(k)
//   adjoint (ADJ = true):  W[i][k] = c_k * sum_q ubar_iq e^{-2 pi i k q/n},
//                          c_0 = c_L = 1, else 2  (transpose of rows_inverse)
//   zonal (optional, FP32 arithmetic): Z[i][0] = the k = 0 value of row i
//   (row_scale[i] * sum_q f_iq, or sum_q ubar_iq), summed in double-float from
//   the double inputs, Z[i][1] = 0; the FP64 side path takes the zonal column
//   from there.
// One tile = `rows` consecutive rows; shared memory rows * L complex.
// ---------------------------------------------------------------------------
template <typename T, bool ADJ, typename Src>
__device__ __forceinline__ void rows_forward_load(int row0, cpx<T>* __restrict__ sm, const Src& src, int nt,
    int n, int rows, const int* __restrict__ perm, const double* __restrict__ row_scale,
    cpx<double>* __restrict__ zonal) {
  const int L = n >> 1;
  for (int r = 0; r < rows; ++r) {
    const int row = row0 + r;
    dd acc(0.f, 0.f);
#pragma unroll (sizeof(T) == 4 ? 8 : 4)
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
      cpx<T> z = {(T)0, (T)0};
      if (row < nt) {
        double2 v = src(r, q);
        z = {load_conv<T>(v.x), load_conv<T>(v.y)};
        if (zonal) acc = dd_add(acc, dd_add(split_double(v.x), split_double(v.y)));
      }
      sm[r * L + __ldg(perm + q)] = z;
    }
    if (zonal) {  // uniform over the block
      dd tot = block_sum_dd(acc);
      if (threadIdx.x == 0 && row < nt) {
        double g0 = dd_to_double(tot);
        if (!ADJ) g0 *= __ldg(row_scale + row);
        zonal[(size_t)row * 2] = {g0, 0.0};
        zonal[(size_t)row * 2 + 1] = {0.0, 0.0};
      }
    }
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void rows_forward_finish(int row0, cpx<T>* __restrict__ sm, cpx<T>* __restrict__ W,
    int nt, int n, int Kp, int rows, const FftDesc& d, const cpx<T>* __restrict__ tw,
    const cpx<T>* __restrict__ post, const T* __restrict__ row_scale_t) {
  const int L = n >> 1;
  fft_run<-1, BIG>(sm, rows, d, tw);
  const int K = L + 1;
  for (int r = 0; r < rows; ++r) {
   const int row = row0 + r;
   if (row >= nt) break;
   const T hrs = ADJ ? (T)1 : (T)0.5 * row_scale_t[row];   // half the row scale
   cpx<T>* Wr = W + (size_t)row * Kp;
   const cpx<T>* Z = sm + r * L;
   // outputs k and L - k together: with A = Z_k + conj(Z_{L-k}), D = Z_k - conj(Z_{L-k})
   // and e = exp(-2 pi i k/n), G_k = s (A - i e D) and, since the pair's A, D are
   // conj(A), -conj(D) and its e is -conj(e), G_{L-k} = s conj(A + i e D)
   for (int k = threadIdx.x; k <= L / 2; k += blockDim.x) {
      const cpx<T> zk = Z[k];
      const cpx<T> zc = conj(Z[k == 0 ? 0 : L - k]);
      const cpx<T> e = ldg_c(post + k);           // exp(-2 pi i k / n)
      const cpx<T> A = zk + zc, D = zk - zc;
      const T x1 = fma(e.re, D.im, e.im * D.re), x2 = fma(e.re, D.re, -(e.im * D.im));   // e D = x2 + i x1
      const T hs = ADJ ? (k == 0 ? (T)0.5 : (T)1) : hrs;
      // the scale taken into the final FMAs: s (A.re + x1) = fma(s, x1, s A.re), ...
      const cpx<T> hA = {hs * A.re, hs * A.im};
      Wr[k] = {fma(hs, x1, hA.re), fma(-hs, x2, hA.im)};
      const int kk = L - k;
      if (kk != k) Wr[kk] = {fma(-hs, x1, hA.re), fma(-hs, x2, -hA.im)};
   }
   for (int k = K + threadIdx.x; k < Kp; k += blockDim.x) Wr[k] = {(T)0, (T)0};
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void rows_forward_tile(int tile, cpx<T>* __restrict__ sm,
    const double* __restrict__ f, cpx<T>* __restrict__ W, int nt, int n, int Kp, int rows,
    const FftDesc& d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, cpx<double>* __restrict__ zonal) {
  const int row0 = tile * rows;
  const FromInput src{reinterpret_cast<const double2*>(f) + (size_t)row0 * (n >> 1), (size_t)(n >> 1)};
  rows_forward_load<T, ADJ>(row0, sm, src, nt, n, rows, perm, row_scale, zonal);
  __syncthreads();
  rows_forward_finish<T, ADJ, BIG>(row0, sm, W, nt, n, Kp, rows, d, tw, post, row_scale_t);
}

// FP32 longitude kernels are bounded to 40 registers (small spills): five
// 256-thread CTAs then fit per SM (their 40 KB of shared memory allows five)
// instead of four, which took the forward kernel 0.306 -> 0.281 ms at
// 5000 x 10000.  The FP64 transforms also come as the *_two kernels at the
// end of this file, bounded to two 512-thread CTAs per SM.
template <typename T, bool ADJ, bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512, (sizeof(T) == 4 && !BIG) ? 3 : 1) k_rows_forward(
    const double* __restrict__ f, cpx<T>* __restrict__ W, int nt, int n, int Kp, int rows,
    FftDesc d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, cpx<double>* __restrict__ zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  rows_forward_tile<T, ADJ, BIG>(blockIdx.x, sm, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}

// Pipelined form: a persistent CTA loops over tiles blockIdx.x, + gridDim.x,
// ...; while tile t is transformed in the FFT buffer, cp.async stages the
// input rows of the CTA's next tile in a second shared-memory buffer (rows * n
// doubles after the rows * L complex FFT buffer), so HBM reads overlap the
// arithmetic of the same CTA.
template <typename T, bool ADJ>
__global__ void __launch_bounds__(512) k_rows_forward_pipe(
    const double* __restrict__ f, cpx<T>* __restrict__ W, int nt, int n, int Kp, int rows,
    FftDesc d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, cpx<double>* __restrict__ zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = n >> 1;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  double2* S = reinterpret_cast<double2*>(smem_raw + (((size_t)rows * L * sizeof(cpx<T>) + 15) & ~(size_t)15));
  const int ntiles = (nt + rows - 1) / rows;
  auto stage = [&](int t) {
    const int row0 = t * rows;
    stage_rows<16>(S, f + (size_t)row0 * n, (size_t)n * sizeof(double), min(rows, nt - row0),
                   n * (int)sizeof(double));
  };
  int tile = blockIdx.x;
  if (tile < ntiles) stage(tile);
  cp_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    cp_wait_all();
    __syncthreads();
    const int row0 = tile * rows;
    rows_forward_load<T, ADJ>(row0, sm, FromStaged<double2>{S, L}, nt, n, rows, perm, row_scale, zonal);
    __syncthreads();
    if (tile + (int)gridDim.x < ntiles) stage(tile + gridDim.x);
    cp_commit();
    rows_forward_finish<T, ADJ, false>(row0, sm, W, nt, n, Kp, rows, d, tw, post, row_scale_t);
  }
  cp_wait_all();
}

// ---------------------------------------------------------------------------
// rows_inverse: inverse real FFT along longitude,
//   u_iq = Re U_0 + 2 Re sum_{k=1}^{L-1} U_k e^{2 pi i k q/n} + Re U_L (-1)^q.
//   forward: U = W, u written unscaled.
//   adjoint: U_k = W_k * (k == 0 || k == L ? 1 : 1/2), u scaled by row_scale
//            (transpose of rows_forward).
//   zonal (optional): U_0 of row i is taken as Z[i][0].re, added in double
//            after the transform (the FP64 side path's zonal column).
// ---------------------------------------------------------------------------
template <typename T, bool ADJ, typename Src>
__device__ __forceinline__ void rows_inverse_load(int row0, cpx<T>* __restrict__ sm, const Src& src, int nt,
    int n, int rows, const int* __restrict__ perm, const cpx<T>* __restrict__ post, bool zonal) {
  const int L = n >> 1;
  // inputs k and L - k together: with A = U_k + conj(U_{L-k}), D = U_k - conj(U_{L-k})
  // and e = exp(-2 pi i k/n), Z_k = A + i conj(e) D and, since the pair's A, D
  // are conj(A), -conj(D) and its e is -conj(e), Z_{L-k} = conj(A) + i e conj(D)
  // (k = 0 pairs with the Nyquist bin U_L and has no partner)
  for (int r = 0; r < rows; ++r)
#pragma unroll 2
  for (int k = threadIdx.x; k <= L / 2; k += blockDim.x) {
    const int row = row0 + r;
    const int kk = L - k;
    cpx<T> z = {(T)0, (T)0}, zp = {(T)0, (T)0};
    if (row < nt) {
      cpx<T> uk = src(r, k);
      cpx<T> up = src(r, kk);
      if (k == 0) {
        uk.im = (T)0;
        up.im = (T)0;
        if (zonal) uk.re = (T)0;
      } else if (ADJ) {
        uk = (T)0.5 * uk;
        up = (T)0.5 * up;
      }
      const cpx<T> uc = conj(up);
      const cpx<T> e = ldg_c(post + k);          // conj(e) = exp(+2 pi i k / n)
      const cpx<T> A = uk + uc, D = uk - uc;
      const T x1 = fma(e.re, D.im, -(e.im * D.re)), x2 = fma(e.re, D.re, e.im * D.im);
      z = {A.re - x1, A.im + x2};
      zp = {A.re + x1, x2 - A.im};
    }
    sm[r * L + __ldg(perm + k)] = z;
    if (k != 0 && kk != k) sm[r * L + __ldg(perm + kk)] = zp;
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void rows_inverse_finish(int row0, cpx<T>* __restrict__ sm, double* __restrict__ u,
    int nt, int n, int rows, const FftDesc& d, const cpx<T>* __restrict__ tw,
    const double* __restrict__ row_scale, const T* __restrict__ row_scale_t,
    const cpx<double>* __restrict__ zonal) {
  const int L = n >> 1;
  fft_run<+1, BIG>(sm, rows, d, tw);
  for (int r = 0; r < rows; ++r)
  for (int q = threadIdx.x; q < L; q += blockDim.x) {
    const int row = row0 + r;
    if (row >= nt) break;
    cpx<T> z = sm[r * L + q];
    double2 v;
    if constexpr (std::is_same<T, double>::value) {
      double scale = ADJ ? __ldg(row_scale + row) : 1.0;
      v = {scale * z.re, scale * z.im};
    } else {
      // reduced-precision forms: the zonal value is added, and the adjoint's row
      // scale applied, in the transform's arithmetic before widening to double
      if (zonal) {
        T u0 = load_conv<T>(zonal[(size_t)row * 2].re);
        z = {z.re + u0, z.im + u0};
      }
      if (ADJ) z = row_scale_t[row] * z;
      v = {store_conv<T>(z.re), store_conv<T>(z.im)};
    }
    reinterpret_cast<double2*>(u + (size_t)row * n)[q] = v;
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void rows_inverse_tile(int tile, cpx<T>* __restrict__ sm,
    const cpx<T>* __restrict__ W, double* __restrict__ u, int nt, int n, int Kp, int rows,
    const FftDesc& d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, const cpx<double>* __restrict__ zonal) {
  const int row0 = tile * rows;
  rows_inverse_load<T, ADJ>(row0, sm, FromGlobal<cpx<T>>{W + (size_t)row0 * Kp, (size_t)Kp}, nt, n, rows, perm,
                            post, zonal != nullptr);
  __syncthreads();
  rows_inverse_finish<T, ADJ, BIG>(row0, sm, u, nt, n, rows, d, tw, row_scale, row_scale_t, zonal);
}

template <typename T, bool ADJ, bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512, (sizeof(T) == 4 && !BIG) ? 3 : 1) k_rows_inverse(
    const cpx<T>* __restrict__ W, double* __restrict__ u, int nt, int n, int Kp, int rows,
    FftDesc d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, const cpx<double>* __restrict__ zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  rows_inverse_tile<T, ADJ, BIG>(blockIdx.x, sm, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t, zonal);
}

// pipelined form (see k_rows_forward_pipe): the staged copy holds the tile's
// spectrum rows, rows * Kp complex T, after the rows * L FFT buffer
template <typename T, bool ADJ>
__global__ void __launch_bounds__(512) k_rows_inverse_pipe(
    const cpx<T>* __restrict__ W, double* __restrict__ u, int nt, int n, int Kp, int rows,
    FftDesc d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, const cpx<double>* __restrict__ zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = n >> 1;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw + (((size_t)rows * L * sizeof(cpx<T>) + 15) & ~(size_t)15));
  const int ntiles = (nt + rows - 1) / rows;
  auto stage = [&](int t) {
    const int row0 = t * rows;
    stage_rows<16>(S, W + (size_t)row0 * Kp, (size_t)Kp * sizeof(cpx<T>), min(rows, nt - row0),
                   Kp * (int)sizeof(cpx<T>));
  };
  int tile = blockIdx.x;
  if (tile < ntiles) stage(tile);
  cp_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    cp_wait_all();
    __syncthreads();
    const int row0 = tile * rows;
    rows_inverse_load<T, ADJ>(row0, sm, FromStaged<cpx<T>>{S, Kp}, nt, n, rows, perm, post, zonal != nullptr);
    __syncthreads();
    if (tile + (int)gridDim.x < ntiles) stage(tile + gridDim.x);
    cp_commit();
    rows_inverse_finish<T, ADJ, false>(row0, sm, u, nt, n, rows, d, tw, row_scale, row_scale_t, zonal);
  }
  cp_wait_all();
}

// ---------------------------------------------------------------------------
// theta_forward: per column k, P_j = (1/2)(w_j V_j + conj(w_j) V_{N-j}), with
// V = FFT_N of the Makhoul-reordered column (odd k: samples times (-1)^i) and
// w_j = exp(-i pi j / (2N)); P is DCT-II of the column (odd k: P_{N-j} is its
// DST-II at j).
//   forward: F_j = P_j / N (k even), F_j = -i P_{N-j} / N (k odd, F_0 = 0)
//   adjoint: Xbar_j = c_j P_j (k even, c_0 = 1, c_j = 2), Xbar_j = -2i P_{N-j}
//            (k odd, Xbar_0 = 0)  (transpose of theta_inverse); with bit 1 of
//            `zonal` set (FP64 arithmetic), column 0 also gets the transposed
//            k = 0 closure.
//   bit 2 of `zonal` multiplies the result by (-1)^k: the coefficients of the
//   paper's expansion in e^{i k lambda} with lambda_q = -pi + 2 pi q/n.
// One tile = `cols` consecutive columns.  inv_n = 1/N in arithmetic T.
// ---------------------------------------------------------------------------
template <typename T, typename Src>
__device__ __forceinline__ void theta_forward_load(int k0, cpx<T>* __restrict__ sm, const Src& src, int N,
                                                   int K, int cols, const int* __restrict__ perm) {
  const int cs = __ffs(cols) - 1;            // cols is a power of two
#pragma unroll 4
  for (int idx = threadIdx.x; idx < N * cols; idx += blockDim.x) {
    int i = idx >> cs, c = idx & (cols - 1);
    int k = k0 + c;
    cpx<T> v = {(T)0, (T)0};
    if (k < K) {
      v = neg_if(src(i, c), (k & 1) && (i & 1));
    }
    sm[c * N + __ldg(perm + makhoul_pos(i, N))] = v;
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void theta_forward_finish(int k0, cpx<T>* __restrict__ sm, cpx<T>* __restrict__ W,
    int N, int K, int Kp, int cols, const FftDesc& d, const cpx<T>* __restrict__ tw,
    const cpx<T>* __restrict__ post, int zonal) {
  const int cs = __ffs(cols) - 1;
  fft_run<-1, BIG>(sm, cols, d, tw);
  // P_j = w_j V_j + conj(w_j) V_{N-j} (the forward passes the table w/(2N), the
  // adjoint w itself) for the pair j, N - j at once: with S = V_j + V_{N-j},
  // D = V_j - V_{N-j} and w_{N-j} = -i conj(w_j),
  //   P_j = (w.re S.re - w.im D.im, w.re S.im + w.im D.re),
  //   P_{N-j} = (-w.im S.re - w.re D.im, -w.im S.im + w.re D.re).
  // k even: F_j = P_j; k odd: F_j = -i P_{N-j} (F_0 = 0).
  const int H = N / 2 + 1;
  for (int idx = threadIdx.x; idx < H * cols; idx += blockDim.x) {
    const int j = idx >> cs, c = idx & (cols - 1);
    const int k = k0 + c;
    if (k >= K) continue;
    const cpx<T>* V = sm + c * N;
    const int jj = N - j;                      // partner output (none for j = 0, or jj = j)
    const bool pair = j > 0 && jj != j;
    const cpx<T> w = ldg_c(post + j);
    const cpx<T> a = V[j], b = V[j == 0 ? 0 : jj];
    const cpx<T> S = a + b, D = a - b;
    const cpx<T> pj = {fma(w.re, S.re, -(w.im * D.im)), fma(w.re, S.im, w.im * D.re)};
    const cpx<T> pjj = {fma(-w.im, S.re, -(w.re * D.im)), fma(-w.im, S.im, w.re * D.re)};
    cpx<T>* out = W + k;
    if ((k & 1) == 0) {
      cpx<T> oj = pj, ojj = pjj;
      if (ADJ) {
        if (j == 0) oj = (T)0.5 * oj;
        if constexpr (std::is_same<T, double>::value) {
          // transpose of the k = 0 closure X_0 = sum_{j even >= 2} 2 X_j/(j^2-1):
          // Xbar_j += 2 Xbar_0/(j^2-1), with Xbar_0 = P_0 = V_0
          if ((zonal & 1) && k == 0) {
            if (j >= 2 && !(j & 1)) oj = oj + (2.0 / ((double)j * (double)j - 1.0)) * V[0];
            if (jj >= 2 && !(jj & 1)) ojj = ojj + (2.0 / ((double)jj * (double)jj - 1.0)) * V[0];
          }
        }
      }
      out[(size_t)j * Kp] = oj;
      if (pair) out[(size_t)jj * Kp] = ojj;
    } else {
      // -i p, times -1 in the coefficient convention ((-1)^k for k odd)
      const bool ng = (zonal & 2) != 0;
      out[(size_t)j * Kp] = j == 0 ? cpx<T>{(T)0, (T)0} : cpx<T>{neg_if(pjj.im, ng), neg_if(pjj.re, !ng)};
      if (pair) out[(size_t)jj * Kp] = {neg_if(pj.im, ng), neg_if(pj.re, !ng)};
    }
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void theta_forward_tile(int tile, cpx<T>* __restrict__ sm,
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, const FftDesc& d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  (void)inv_n;
  const int k0 = tile * cols;
  theta_forward_load<T>(k0, sm, FromGlobal<cpx<T>>{W + k0, (size_t)Kp}, N, K, cols, perm);
  __syncthreads();
  theta_forward_finish<T, ADJ, BIG>(k0, sm, W, N, K, Kp, cols, d, tw, post, zonal);
}

template <typename T, bool ADJ, bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_forward(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  theta_forward_tile<T, ADJ, BIG>(blockIdx.x, sm, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}

// cp.async staging of the columns [k0, k0 + cols) of all N rows of W into S
// (N rows of `cols` elements; columns at or past Kp are not copied, and the
// loaders never read them since K <= Kp)
template <typename T>
__device__ __forceinline__ void stage_theta(cpx<T>* S, const cpx<T>* W, int k0, int N, int Kp, int cols) {
  const int ncols = min(cols, Kp - k0);
  const int row_bytes = cols * (int)sizeof(cpx<T>);
  const size_t ld = (size_t)Kp * sizeof(cpx<T>);
  if ((ncols * sizeof(cpx<T>)) % 16 == 0) {
    const int per = ncols * (int)sizeof(cpx<T>) / 16;
    const int slots = cols * (int)sizeof(cpx<T>) / 16;      // a power of two >= per
    stage_columns<16>(S, W + k0, ld, N, __ffs(slots) - 1, per, row_bytes);
  } else {                                   // one FP32 complex per row
    stage_columns<8>(S, W + k0, ld, N, 0, 1, row_bytes);
  }
}

// pipelined form: persistent CTAs, the next tile's columns staged by cp.async
// (N * cols complex T after the cols * N FFT buffer) during the transform
template <typename T, bool ADJ>
__global__ void __launch_bounds__(512) k_theta_forward_pipe(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  (void)inv_n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw + (((size_t)cols * N * sizeof(cpx<T>) + 15) & ~(size_t)15));
  const int ntiles = (K + cols - 1) / cols;
  int tile = blockIdx.x;
  if (tile < ntiles) stage_theta(S, W, tile * cols, N, Kp, cols);
  cp_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    cp_wait_all();
    __syncthreads();
    const int k0 = tile * cols;
    theta_forward_load<T>(k0, sm, FromStaged<cpx<T>>{S, cols}, N, K, cols, perm);
    __syncthreads();
    if (tile + (int)gridDim.x < ntiles) stage_theta(S, W, (tile + gridDim.x) * cols, N, Kp, cols);
    cp_commit();
    theta_forward_finish<T, ADJ, false>(k0, sm, W, N, K, Kp, cols, d, tw, post, zonal);
  }
  cp_wait_all();
}

// ---------------------------------------------------------------------------
// theta_inverse: per column k, DCT-III (k even) U_i = Y_0 + 2 sum_j Y_j cos(j theta_i)
// with Y = X, or for k odd i (-1)^i times the DCT-III of Y_j = X_{N-j} (Y_0 = 0),
// through one inverse FFT of V_j = exp(i pi j/(2N)) (Y_j - i Y_{N-j}) (Y_N = 0)
// and the inverse Makhoul reordering.
//   forward: U = DCT-III(X) (k even), i DST-III(X) (k odd); with bit 1 of
//            `zonal` set (FP64 arithmetic) the first tile first closes the
//            k = 0 column: X_00 = sum_{j even >= 2} 2 X_j0/(j^2-1) (w^T X_0 = 0);
//            bit 2 takes the input in the coefficient convention (times (-1)^k).
//   adjoint: inputs with j >= 1 halved and outputs scaled by inv_n = 1/N: the
//            transpose of theta_forward
// ---------------------------------------------------------------------------
// the k = 0 closure of the FP64 path (whole CTA; W[0] written)
__device__ __forceinline__ void zonal_closure(cpx<double>* __restrict__ W, int N, int Kp) {
  cpx<double> acc = {0.0, 0.0};
  for (int j = 2 + 2 * threadIdx.x; j < N; j += 2 * blockDim.x) {
    double wj = 2.0 / ((double)j * (double)j - 1.0);
    acc = acc + wj * W[(size_t)j * Kp];
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc.re = acc.re + __shfl_down_sync(0xffffffffu, acc.re, off);
    acc.im = acc.im + __shfl_down_sync(0xffffffffu, acc.im, off);
  }
  __shared__ cpx<double> red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    cpx<double> tot = {0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot = tot + red[w];
    W[0] = tot;
  }
  __syncthreads();
}

template <typename T, bool ADJ, typename Src>
__device__ __forceinline__ void theta_inverse_load(int k0, cpx<T>* __restrict__ sm, const Src& src, int N,
    int K, int cols, const int* __restrict__ perm, const cpx<T>* __restrict__ post, int zonal) {
  // pre-twiddle, one thread per pair (j, N - j), j = 0 .. N/2, writing V_j and
  // V_{N-j} to their digit-reversed slots
  const int H = N / 2 + 1;
  const int cs = __ffs(cols) - 1;            // cols is a power of two
#pragma unroll 2
  for (int idx = threadIdx.x; idx < H * cols; idx += blockDim.x) {
    int j = idx >> cs, c = idx & (cols - 1);
    int k = k0 + c;
    cpx<T>* V = sm + c * N;
    const bool odd = (k & 1);
    if (k >= K) {
      V[__ldg(perm + j)] = {(T)0, (T)0};
      if (j > 0 && N - j != j) V[__ldg(perm + N - j)] = {(T)0, (T)0};
      continue;
    }
    if (j == 0) {
      // V_0 = Y_0 - i Y_N = X_0 (k even) or 0 (k odd)
      V[__ldg(perm + 0)] = odd ? cpx<T>{(T)0, (T)0} : src(0, c);
      continue;
    }
    int jj = N - j;
    cpx<T> xa = src(j, c), xb = src(jj, c);
    if (ADJ) {
      xa = (T)0.5 * xa;
      xb = (T)0.5 * xb;
    }
    const bool ng = (zonal & 2) && odd;        // input in the coefficient convention
    xa = neg_if(xa, ng);
    xb = neg_if(xb, ng);
    // Y_j, Y_{N-j}
    cpx<T> ya = odd ? xb : xa;
    cpx<T> yb = odd ? xa : xb;
    cpx<T> wa = conj(ldg_c(post + j));     // exp(+i pi j/(2N))
    V[__ldg(perm + j)] = cmul(wa, cpx<T>{ya.re + yb.im, ya.im - yb.re});   // w (Y_j - i Y_{N-j})
    if (jj != j) {
      cpx<T> wb = conj(ldg_c(post + jj));
      V[__ldg(perm + jj)] = cmul(wb, cpx<T>{yb.re + ya.im, yb.im - ya.re});
    }
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void theta_inverse_finish(int k0, cpx<T>* __restrict__ sm, cpx<T>* __restrict__ W,
    int N, int K, int Kp, int cols, const FftDesc& d, const cpx<T>* __restrict__ tw, T inv_n) {
  const int cs = __ffs(cols) - 1;
  fft_run<+1, BIG>(sm, cols, d, tw);
  for (int idx = threadIdx.x; idx < N * cols; idx += blockDim.x) {
    int i = idx >> cs, c = idx & (cols - 1);
    int k = k0 + c;
    if (k >= K) continue;
    cpx<T> v = sm[c * N + makhoul_pos(i, N)];
    if (ADJ) v = inv_n * v;
    if (k & 1) {
      // times i (-1)^i
      v = {neg_if(v.im, !(i & 1)), neg_if(v.re, (i & 1) != 0)};
    }
    W[(size_t)i * Kp + k] = v;
  }
}

template <typename T, bool ADJ, bool BIG>
__device__ __forceinline__ void theta_inverse_tile(int tile, cpx<T>* __restrict__ sm,
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, const FftDesc& d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  const int k0 = tile * cols;
  if constexpr (std::is_same<T, double>::value) {
    if (!ADJ && (zonal & 1) && k0 == 0) zonal_closure(W, N, Kp);
  }
  theta_inverse_load<T, ADJ>(k0, sm, FromGlobal<cpx<T>>{W + k0, (size_t)Kp}, N, K, cols, perm, post, zonal);
  __syncthreads();
  theta_inverse_finish<T, ADJ, BIG>(k0, sm, W, N, K, Kp, cols, d, tw, inv_n);
}

template <typename T, bool ADJ, bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_inverse(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  theta_inverse_tile<T, ADJ, BIG>(blockIdx.x, sm, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}

// pipelined form (see k_theta_forward_pipe); the CTA that owns tile 0 closes
// the k = 0 column before staging it
template <typename T, bool ADJ>
__global__ void __launch_bounds__(512) k_theta_inverse_pipe(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw + (((size_t)cols * N * sizeof(cpx<T>) + 15) & ~(size_t)15));
  const int ntiles = (K + cols - 1) / cols;
  int tile = blockIdx.x;
  if constexpr (std::is_same<T, double>::value) {
    if (!ADJ && (zonal & 1) && tile == 0) zonal_closure(W, N, Kp);
  }
  if (tile < ntiles) stage_theta(S, W, tile * cols, N, Kp, cols);
  cp_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    cp_wait_all();
    __syncthreads();
    const int k0 = tile * cols;
    theta_inverse_load<T, ADJ>(k0, sm, FromStaged<cpx<T>>{S, cols}, N, K, cols, perm, post, zonal);
    __syncthreads();
    if (tile + (int)gridDim.x < ntiles) stage_theta(S, W, (tile + gridDim.x) * cols, N, Kp, cols);
    cp_commit();
    theta_inverse_finish<T, ADJ, false>(k0, sm, W, N, K, Kp, cols, d, tw, inv_n);
  }
  cp_wait_all();
}

// ---------------------------------------------------------------------------
// Plan-time factorisation of the parity tridiagonals of every column.
// Chain rows j = j0, j0+2, ... < N (j0 = 1 odd chain, 2 even chain), t = 0..M-1:
//   a_j = (j-1)(j-2)/4 (couples j-2), b_j = -(j^2/2 + k^2), c_j = (j+1)(j+2)/4.
// TWIST = false: Thomas without pivoting in increasing j: u_0 = b_j0,
//   l_t = a_t / u_{t-1}, u_t = b_t - l_t c_{t-1}; stored per (j, k): l, 1/u, c/u.
// TWIST = true: a twisted factorisation about the middle row m = (M-1)/2, so
//   that the solve can run the two halves of every chain at once: rows t < m as
//   above; rows t > m eliminated from the bottom, v_{M-1} = b_{M-1},
//   g_t = c_t / v_{t+1}, v_t = b_t - g_t a_{t+1}, stored as g, 1/v, a/v; row m
//   stores l_m = a_m/u_{m-1}, 1/gamma and g_m = c_m/v_{m+1} (in the third table),
//   gamma = b_m - l_m c_{m-1} - g_m a_{m+1}.
// Thread layout: idx < K -> odd chain of k = idx; else even chain of k = idx - K.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double chain_a(double j) { return (j - 1.0) * (j - 2.0) * 0.25; }
__device__ __forceinline__ double chain_c(double j) { return (j + 1.0) * (j + 2.0) * 0.25; }

template <typename S, bool TWIST>
__global__ void k_factor(S* __restrict__ fl, S* __restrict__ fiu, S* __restrict__ fcu,
                         int N, int K, int Kp) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * K) return;
  const bool even = idx >= K;
  const int k = even ? idx - K : idx;
  const double k2 = (double)k * (double)k;
  const int j0 = even ? 2 : 1;
  if (j0 >= N) return;
  const int M = (N - 1 - j0) / 2 + 1;
  const int m = TWIST ? (M - 1) / 2 : M;
  auto row = [&](int t) { return (size_t)(j0 + 2 * t) * Kp + k; };
  auto b_of = [&](int t) { const double j = (double)(j0 + 2 * t); return -(j * j * 0.5 + k2); };
  double u_prev = 0.0, c_prev = 0.0;
  for (int t = 0; t < m; ++t) {
    const double jd = (double)(j0 + 2 * t);
    const double a = chain_a(jd), b = b_of(t), c = chain_c(jd);
    double l = 0.0, uu = b;
    if (t > 0) {
      l = a / u_prev;
      uu = b - l * c_prev;
    }
    const double iu = 1.0 / uu;
    fl[row(t)] = (S)l;
    fiu[row(t)] = (S)iu;
    fcu[row(t)] = (S)(c * iu);
    u_prev = uu;
    c_prev = c;
  }
  if (!TWIST) return;
  double v_next = 0.0, a_next = 0.0;
  for (int t = M - 1; t > m; --t) {
    const double jd = (double)(j0 + 2 * t);
    const double a = chain_a(jd), b = b_of(t), c = chain_c(jd);
    double g = 0.0, vv = b;
    if (t < M - 1) {
      g = c / v_next;
      vv = b - g * a_next;
    }
    const double iv = 1.0 / vv;
    fl[row(t)] = (S)g;
    fiu[row(t)] = (S)iv;
    fcu[row(t)] = (S)(a * iv);
    v_next = vv;
    a_next = a;
  }
  const double jm = (double)(j0 + 2 * m);
  const double lm = m > 0 ? chain_a(jm) / u_prev : 0.0;
  const double gm = m < M - 1 ? chain_c(jm) / v_next : 0.0;
  const double gam = b_of(m) - (m > 0 ? lm * c_prev : 0.0) - (m < M - 1 ? gm * a_next : 0.0);
  fl[row(m)] = (S)lm;
  fiu[row(m)] = (S)(1.0 / gam);
  fcu[row(m)] = (S)gm;
}

// ---------------------------------------------------------------------------
// solve (ADJ = false): X = M_k^{-1} F per column, in place.
//   chains: y_t = d_t - l_t y_{t-1}; x_t = y_t/u_t - (c_t/u_t) x_{t+1}
//   closure (even-chain thread): k even != 0: X_0 = (X_2 - F_0)/k^2 (row 0 with
//   X_{-2,k} = X_{2,k}); k odd: X_0 = 0.  For k = 0, w^T X_0 = 0 with
//   X_{-j,0} = X_{j,0} gives X_0 = sum_{j even >= 2} 2 X_j/(j^2-1), summed by
//   the first CTA of theta_inverse.
// solve (ADJ = true): the transpose, F = M_k^{-T} X:
//   k even != 0: Fbar_0 = -Xbar_0/k^2 and Xbar_2 += Xbar_0/k^2; k = 0:
//   Xbar_j += 2 Xbar_0/(j^2-1) for even j (added by theta_forward's adjoint),
//   Fbar_0 = 0; k odd: Fbar_0 = 0;
//   then the transposed chain solve (below).
// ---------------------------------------------------------------------------
// cp.async helpers (per-thread asynchronous global -> shared copies)

// Each lane streams its own chain's rows through a ring of shared-memory slots
// filled by its own cp.async copies, a ring's depth of rows ahead of the
// elimination, so every lane keeps that many rows of loads in flight without
// any cross-lane synchronisation.
// S is the storage and arithmetic type (double, or float for the FP32 form).
template <typename S>
struct RingSlot {
  cpx<S> d[32];
  S a[32];
  S b[32];
};

template <typename S>
__device__ __forceinline__ void cp_async_c(cpx<S>* smem, const cpx<S>* g) {
  if constexpr (sizeof(cpx<S>) == 16) cp_async16(smem, g);
  else cp_async8(smem, g);
}
template <typename S>
__device__ __forceinline__ void cp_async_s(S* smem, const S* g) {
  if constexpr (sizeof(S) == 8) {
    cp_async8(smem, g);
  } else {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
  }
}

// Rows t = t0 + dir s, s = 0..len-1, of one chain streamed through this warp's
// ring: the copies of row s + kSolveRing are issued after row s has been consumed by
// body(t, d, a, b) (d from Wc, a and b from the tables ta, tb; tb may be null).
// The ring holds kSolveRing rows (two rings of 16 KB each for FP64).
constexpr int kSolveRing = 16;
template <typename S, typename Body>
__device__ __forceinline__ void ring_sweep(RingSlot<S>* ring, int lane, bool active, cpx<S>* Wc, const S* ta,
                                           const S* tb, size_t stride, int t0, int dir, int len, Body body) {
  auto issue = [&](int q) {
    if (active && q < len) {
      const int t = t0 + dir * q;
      RingSlot<S>& sl = ring[q & (kSolveRing - 1)];
      cp_async_c(&sl.d[lane], Wc + t * stride);
      cp_async_s(&sl.a[lane], ta + t * stride);
      if (tb) cp_async_s(&sl.b[lane], tb + t * stride);
    }
    cp_commit();
  };
  for (int q = 0; q < kSolveRing; ++q) issue(q);
  for (int q = 0; q < len; ++q) {
    cp_wait<kSolveRing - 1>();
    const RingSlot<S>& sl = ring[q & (kSolveRing - 1)];
    if (active) body(t0 + dir * q, sl.d[lane], sl.a[lane], tb ? sl.b[lane] : (S)0);
    issue(q + kSolveRing);
  }
  cp_wait_all();
}

// Twisted solve: CTA = 2 warps over the same 32 chains (consecutive k, one
// parity, blockIdx.y = 1 the even chains); warp 0 runs rows t < m from the top,
// warp 1 rows t > m from the bottom, each through its own ring, and they meet
// at the middle row m through shared memory (tables of k_factor<S, true>).
//   forward: y_t = d_t - l_t y_{t-1} (t < m), z_t = d_t - g_t z_{t+1} (t > m),
//     x_m = (d_m - l_m y_{m-1} - g_m z_{m+1}) / gamma, then
//     x_t = y_t/u_t - (c_t/u_t) x_{t+1} (t < m), x_t = z_t/v_t - (a_t/v_t) x_{t-1} (t > m).
//   adjoint (the transpose of those steps in reverse order):
//     p_t = (b_t - c_{t-1} p_{t-1})/u_t (t < m), q_t = (b_t - a_{t+1} q_{t+1})/v_t (t > m),
//     s = (b_m - c_{m-1} p_{m-1} - a_{m+1} q_{m+1}) / gamma, then
//     r_t = p_t - l_{t+1} r_{t+1} (t < m, r_m = s), w_t = q_t - g_{t-1} w_{t-1} (t > m, w_m = s).
constexpr int kSolveThreads = 64;
template <bool ADJ, typename S>
__global__ void __launch_bounds__(kSolveThreads) k_solve(cpx<S>* __restrict__ W, const S* __restrict__ fl,
                                                         const S* __restrict__ fiu, const S* __restrict__ fcu,
                                                         int N, int K, int Kp) {
  __shared__ RingSlot<S> ring[2][kSolveRing];
  __shared__ cpx<S> meet[3][32];
  const int lane = threadIdx.x & 31, half = threadIdx.x >> 5;   // half 0: top, 1: bottom
  const bool even = blockIdx.y == 1;
  const int k = blockIdx.x * 32 + lane;
  const bool active = k < K;
  const int j0 = even ? 2 : 1;
  const S ik2 = k ? (S)(1.0 / ((double)k * (double)k)) : (S)0;
  if (j0 >= N) {
    // no chain rows; only the closure of row 0 remains (forward: X_0 = -F_0/k^2,
    // adjoint: Fbar_0 = -Xbar_0/k^2, both zero for k = 0 and odd k)
    if (even && half == 0 && active) {
      cpx<S> x0 = W[k];
      W[k] = (k == 0 || (k & 1)) ? cpx<S>{(S)0, (S)0} : (-ik2) * x0;
    }
    return;
  }
  const int M = (N - 1 - j0) / 2 + 1;            // chain length
  const int m = (M - 1) / 2;                     // the rows meet at t = m
  const size_t stride = (size_t)2 * Kp;          // one chain step
  cpx<S>* Wc = W + (size_t)j0 * Kp + (active ? k : 0);
  const S* Lc = fl + (size_t)j0 * Kp + (active ? k : 0);
  const S* IUc = fiu + (size_t)j0 * Kp + (active ? k : 0);
  const S* CUc = fcu + (size_t)j0 * Kp + (active ? k : 0);
  RingSlot<S>* rg = ring[half];
  const int jm = j0 + 2 * m;

  if (!ADJ) {
    // first sweeps: y (top, rows 0..m-1) and z (bottom, rows M-1..m+1)
    cpx<S> e = {(S)0, (S)0};
    if (half == 0) {
      ring_sweep(rg, lane, active, Wc, Lc, (const S*)nullptr, stride, 0, 1, m, [&](int t, cpx<S> d, S l, S) {
        e = {fma(-l, e.re, d.re), fma(-l, e.im, d.im)};
        Wc[t * stride] = e;
      });
    } else {
      ring_sweep(rg, lane, active, Wc, Lc, (const S*)nullptr, stride, M - 1, -1, M - 1 - m,
                 [&](int t, cpx<S> d, S g, S) {
                   e = {fma(-g, e.re, d.re), fma(-g, e.im, d.im)};
                   Wc[t * stride] = e;
                 });
    }
    meet[half][lane] = e;
    __syncthreads();
    if (half == 0 && active) {
      const cpx<S> ym1 = meet[0][lane], zp1 = meet[1][lane], dm = Wc[m * stride];
      const S lm = Lc[m * stride], gm = CUc[m * stride], ig = IUc[m * stride];
      const cpx<S> xm = {ig * (dm.re - lm * ym1.re - gm * zp1.re), ig * (dm.im - lm * ym1.im - gm * zp1.im)};
      Wc[m * stride] = xm;
      meet[2][lane] = xm;
    }
    __syncthreads();
    __threadfence();  // the copies below read rows this thread stored
    cpx<S> x = meet[2][lane];
    if (half == 0) {
      ring_sweep(rg, lane, active, Wc, IUc, CUc, stride, m - 1, -1, m, [&](int t, cpx<S> yv, S iu, S cu) {
        x = {fma(yv.re, iu, -cu * x.re), fma(yv.im, iu, -cu * x.im)};
        Wc[t * stride] = x;
      });
      if (even && k != 0 && active) {
        // x holds X_2: row 0 closure X_0 = (X_2 - F_0)/k^2 (k even), X_0 = 0 (k odd).
        // The k = 0 closure (w^T X_0 = 0) is summed by theta_inverse's first CTA.
        cpx<S> f0 = W[k];
        if (k & 1) W[k] = {(S)0, (S)0};
        else W[k] = {(x.re - f0.re) * ik2, (x.im - f0.im) * ik2};
      }
    } else {
      ring_sweep(rg, lane, active, Wc, IUc, CUc, stride, m + 1, 1, M - 1 - m, [&](int t, cpx<S> zv, S iv, S av) {
        x = {fma(zv.re, iv, -av * x.re), fma(zv.im, iv, -av * x.im)};
        Wc[t * stride] = x;
      });
    }
  } else {
    cpx<S> xb0 = {(S)0, (S)0};
    if (even && half == 0 && active) {
      xb0 = W[k];
      W[k] = (k == 0 || (k & 1)) ? cpx<S>{(S)0, (S)0} : (-ik2) * xb0;
    }
    const bool bump2 = even && k != 0 && !(k & 1);   // Xbar_2 += Xbar_0 / k^2 (row t = 0)
    // (k = 0: the terms 2 Xbar_0/(j^2-1) were added by theta_forward's adjoint)
    cpx<S> e = {(S)0, (S)0};
    if (half == 0) {
      ring_sweep(rg, lane, active, Wc, IUc, (const S*)nullptr, stride, 0, 1, m, [&](int t, cpx<S> b, S iu, S) {
        if (bump2 && t == 0) b = {fma(ik2, xb0.re, b.re), fma(ik2, xb0.im, b.im)};
        const int j = j0 + 2 * t;
        const S cprev = t ? (S)((double)((j - 1) * j) * 0.25) : (S)0;   // c_{j-2} = (j-1) j / 4
        e = {(b.re - cprev * e.re) * iu, (b.im - cprev * e.im) * iu};
        Wc[t * stride] = e;
      });
    } else {
      ring_sweep(rg, lane, active, Wc, IUc, (const S*)nullptr, stride, M - 1, -1, M - 1 - m,
                 [&](int t, cpx<S> b, S iv, S) {
                   const int j = j0 + 2 * t;
                   const S anext = t < M - 1 ? (S)((double)((j + 1) * j) * 0.25) : (S)0;   // a_{j+2}
                   e = {(b.re - anext * e.re) * iv, (b.im - anext * e.im) * iv};
                   Wc[t * stride] = e;
                 });
    }
    meet[half][lane] = e;
    __syncthreads();
    if (half == 0 && active) {
      const cpx<S> pm1 = meet[0][lane], qp1 = meet[1][lane];
      cpx<S> bm = Wc[m * stride];
      if (bump2 && m == 0) bm = {fma(ik2, xb0.re, bm.re), fma(ik2, xb0.im, bm.im)};
      const S cm1 = m > 0 ? (S)((double)((jm - 1) * jm) * 0.25) : (S)0;       // c_{jm-2}
      const S ap1 = m < M - 1 ? (S)((double)((jm + 1) * jm) * 0.25) : (S)0;   // a_{jm+2}
      const S ig = IUc[m * stride];
      const cpx<S> sm = {ig * (bm.re - cm1 * pm1.re - ap1 * qp1.re), ig * (bm.im - cm1 * pm1.im - ap1 * qp1.im)};
      Wc[m * stride] = sm;
      meet[2][lane] = sm;
    }
    __syncthreads();
    __threadfence();
    cpx<S> r = meet[2][lane];
    if (half == 0) {
      S lnext = active ? Lc[m * stride] : (S)0;
      ring_sweep(rg, lane, active, Wc, Lc, (const S*)nullptr, stride, m - 1, -1, m, [&](int t, cpx<S> pv, S l, S) {
        r = {fma(-lnext, r.re, pv.re), fma(-lnext, r.im, pv.im)};
        Wc[t * stride] = r;
        lnext = l;
      });
    } else {
      S gprev = active ? CUc[m * stride] : (S)0;
      ring_sweep(rg, lane, active, Wc, Lc, (const S*)nullptr, stride, m + 1, 1, M - 1 - m,
                 [&](int t, cpx<S> qv, S g, S) {
                   r = {fma(-gprev, r.re, qv.re), fma(-gprev, r.im, qv.im)};
                   Wc[t * stride] = r;
                   gprev = g;
                 });
    }
  }
}

// ---------------------------------------------------------------------------
// Zonal column (k = 0) eliminations in FP64 with a parallel scan.  The two
// parity chains (threads [0, T/2) odd, [T/2, T) even) are each a sequence of
// first-order recurrences x_t = alpha_t x_{t-1} + beta_t (ascending) or
// x_t = alpha_t x_{t+1} + beta_t (descending).  Each thread owns a contiguous
// segment of the chain: it composes its segment's affine map (alpha product
// and the image of 0), the maps are combined across the half-block by a
// Hillis-Steele scan in shared memory, and each thread then re-runs its
// segment from the correct incoming value.  Same arithmetic results as the
// sequential sweeps up to rounding order; used where one sequential chain
// would be the critical path (the FP32 forms' FP64 zonal column).
// ---------------------------------------------------------------------------
struct AffineC {
  double a;          // multiplier
  cpx<double> b;     // offset
};

// combine: first `lo` (earlier segment), then `hi`: x -> hi.a (lo.a x + lo.b) + hi.b
__device__ __forceinline__ AffineC affine_then(AffineC lo, AffineC hi) {
  return {hi.a * lo.a, {fma(hi.a, lo.b.re, hi.b.re), fma(hi.a, lo.b.im, hi.b.im)}};
}

// inclusive scan of one affine map per thread over each half of the block;
// returns the composition of all earlier segments (exclusive prefix) of this half
__device__ __forceinline__ AffineC half_block_exclusive_scan(AffineC mine, AffineC* sh) {
  const int half = blockDim.x >> 1;
  const int h = threadIdx.x >= half;
  const int i = threadIdx.x - h * half;
  AffineC* arr = sh + h * half;
  arr[i] = mine;
  __syncthreads();
  for (int off = 1; off < half; off <<= 1) {
    AffineC cur = arr[i];
    AffineC prev = i >= off ? arr[i - off] : AffineC{1.0, {0.0, 0.0}};
    __syncthreads();
    arr[i] = affine_then(prev, cur);
    __syncthreads();
  }
  AffineC ex = i > 0 ? arr[i - 1] : AffineC{1.0, {0.0, 0.0}};
  __syncthreads();
  return ex;
}

// Z [N][2] column 0: forward (ADJ = false) or transposed (ADJ = true) k = 0
// eliminations with the FP64 factors zl, ziu, zcu ([N][2] layout).  Launch
// one CTA with an even number of threads and (threads) AffineC of dynamic
// shared memory.  Row 0 (the closure) is left to the caller's k = 0 closure.
template <bool ADJ>
__global__ void __launch_bounds__(512) k_zonal_scan(cpx<double>* __restrict__ Z, const double* __restrict__ zl,
                                                    const double* __restrict__ ziu,
                                                    const double* __restrict__ zcu, int N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AffineC* sh = reinterpret_cast<AffineC*>(smem_raw);
  const int half = blockDim.x >> 1;
  const bool even = threadIdx.x >= half;
  const int i = threadIdx.x - (even ? half : 0);
  const int j0 = even ? 2 : 1;
  const int M = j0 < N ? (N - 1 - j0) / 2 + 1 : 0;
  const int seg = (M + half - 1) / half;
  const int t_begin = min(M, i * seg), t_end = min(M, t_begin + seg);
  auto row = [&](int t) { return (size_t)(j0 + 2 * t) * 2; };
  // transposed k = 0 closure: Fbar_0 = 0 (its Xbar_0 terms were added by theta_forward)
  if (ADJ && threadIdx.x == 0) Z[0] = {0.0, 0.0};
  // ---- ascending sweep ----
  // forward:  y_t = -l_t y_{t-1} + d_t
  // adjoint:  z_t = -(c_{t-1} u_t^{-1}) z_{t-1} + b_t u_t^{-1}
  auto up_alpha = [&](int t) -> double {
    if (!ADJ) return -zl[row(t)];
    if (t == 0) return 0.0;
    const int j = j0 + 2 * t;
    return -((double)((j - 1) * j) * 0.25) * ziu[row(t)];
  };
  auto up_beta = [&](int t) -> cpx<double> {
    cpx<double> v = Z[row(t)];
    if (!ADJ) return v;
    return ziu[row(t)] * v;
  };
  AffineC m = {1.0, {0.0, 0.0}};
  for (int t = t_begin; t < t_end; ++t) m = affine_then(m, AffineC{up_alpha(t), up_beta(t)});
  AffineC ex = half_block_exclusive_scan(m, sh);
  cpx<double> x = ex.b;  // value entering this segment (chain starts from 0)
  for (int t = t_begin; t < t_end; ++t) {
    double a = up_alpha(t);
    cpx<double> b = up_beta(t);
    x = {fma(a, x.re, b.re), fma(a, x.im, b.im)};
    Z[row(t)] = x;
  }
  __syncthreads();
  // ---- descending sweep (segments mirrored: thread i takes rows from the end) ----
  // forward:  x_t = -(c_t/u_t) x_{t+1} + y_t / u_t
  // adjoint:  y_t = -l_{t+1} y_{t+1} + z_t
  auto dn_alpha = [&](int t) -> double {
    if (!ADJ) return -zcu[row(t)];
    return t + 1 < M ? -zl[row(t + 1)] : 0.0;
  };
  auto dn_beta = [&](int t) -> cpx<double> {
    cpx<double> v = Z[row(t)];
    if (!ADJ) return ziu[row(t)] * v;
    return v;
  };
  const int r_begin = min(M, i * seg), r_end = min(M, r_begin + seg);   // r = M-1-t
  m = {1.0, {0.0, 0.0}};
  for (int r = r_begin; r < r_end; ++r) {
    const int t = M - 1 - r;
    m = affine_then(m, AffineC{dn_alpha(t), dn_beta(t)});
  }
  ex = half_block_exclusive_scan(m, sh);
  x = ex.b;
  for (int r = r_begin; r < r_end; ++r) {
    const int t = M - 1 - r;
    double a = dn_alpha(t);
    cpx<double> b = dn_beta(t);
    x = {fma(a, x.re, b.re), fma(a, x.im, b.im)};
    Z[row(t)] = x;
  }
}


// exact product of two floats holding integers, as double-float (TwoProduct)
__device__ __forceinline__ dd dd_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return dd(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ cpx<dd> cdd_scale(dd s, cpx<dd> x) { return {dd_mul(s, x.re), dd_mul(s, x.im)}; }

#ifdef SP_REFINE_KERNELS  // defined only in the double-float translation unit
// ---------------------------------------------------------------------------
// Iterative refinement of the per-k eliminations (FP32 + refinement form).
// F (double-float) holds the right-hand sides, X (double-float) the current
// solution, Y a float scratch.  One sweep of chain (k >= 1, parity):
//   R_t = F_t - (a_t X_{t-1} + b_t X_t + c_t X_{t+1})   in double-float (FP64-accurate)
//   FP32 Thomas on R with the FP32 factors: y = R - l y_prev; d = y/u - (c/u) d_next
//   X_t += d_t                                            in double-float
// With first = 1, X is taken as zero (R = F): the unrefined FP32 solve.
// The even chain also sets the row 0 closure X_0 = (X_2 - F_0)/k^2 (k even),
// X_0 = 0 (k odd).  Column k = 0 is left to the FP64 zonal path.
// ---------------------------------------------------------------------------
struct RefSlot {
  cpx<dd> f[32];
  cpx<dd> x[32];
  float a[32];
};
struct RefSlotDown {
  cpx<float> y[32];
  cpx<dd> x[32];
  float a[32];
  float b[32];
};
union RefRing {
  RefSlot up[16];
  RefSlotDown down[16];
};
constexpr int kRefRing = 16;
constexpr int kRefineThreads = 64;

// R_t = F_t - (a_t X_{t-1} + b_t X_t + c_t X_{t+1}) in double-float, the
// coefficients exact: a = (j-1)(j-2)/4, b = -(j^2 + 2k^2)/2, c = (j+1)(j+2)/4
__device__ __forceinline__ cpx<dd> refine_residual(cpx<dd> f, float jf, dd two_k2, cpx<dd> xm1, cpx<dd> x0,
                                                   cpx<dd> xp1) {
  dd a = dd_prod(jf - 1.f, jf - 2.f);
  a = dd(a.hi * 0.25f, a.lo * 0.25f);
  dd b = dd_add(dd_prod(jf, jf), two_k2);
  b = dd(b.hi * -0.5f, b.lo * -0.5f);
  dd c = dd_prod(jf + 1.f, jf + 2.f);
  c = dd(c.hi * 0.25f, c.lo * 0.25f);
  cpx<dd> lx = cdd_scale(b, x0);
  lx = {dd_fma(a, xm1.re, lx.re), dd_fma(a, xm1.im, lx.im)};
  lx = {dd_fma(c, xp1.re, lx.re), dd_fma(c, xp1.im, lx.im)};
  return {dd_sub(f.re, lx.re), dd_sub(f.im, lx.im)};
}

// Twisted form (tables of k_factor<float, true>): CTA = 2 warps over the same
// 32 chains; warp 0 takes rows t < m upwards, warp 1 rows t > m downwards, both
// forming residuals and the FP32 elimination of their half into Y; at the middle
// row m (one barrier) warp 0 forms the row's residual and correction
// d_m = (R_m - l_m y_{m-1} - g_m z_{m+1}) / gamma; both then substitute outwards
// (d_t = y_t/u_t - (c_t/u_t) d_{t+1} above, d_t = z_t/v_t - (a_t/v_t) d_{t-1}
// below) and add d to X.  Every read of X precedes the barrier, every write
// follows it.
__global__ void __launch_bounds__(kRefineThreads) k_refine(const cpx<dd>* __restrict__ F, cpx<dd>* __restrict__ X,
                                                           cpx<float>* __restrict__ Y, const float* __restrict__ fl,
                                                           const float* __restrict__ fiu,
                                                           const float* __restrict__ fcu, int N, int K, int Kp,
                                                           int first) {
  __shared__ RefRing rings[2];
  __shared__ cpx<float> meet[3][32];
  const int lane = threadIdx.x & 31, half = threadIdx.x >> 5;
  const bool even = blockIdx.y == 1;
  const int k = blockIdx.x * 32 + lane;
  const bool active = k < K && k != 0;          // column k = 0 is the FP64 zonal path's
  const int j0 = even ? 2 : 1;
  const float kf = (float)k;
  const dd two_k2 = dd_mul(dd_prod(kf, kf), dd(2.f, 0.f));   // 2 k^2, exact
  RefRing& ring = rings[half];
  const cpx<dd> zero = {dd(0.f, 0.f), dd(0.f, 0.f)};
  if (j0 < N) {
    const int M = (N - 1 - j0) / 2 + 1;
    const int m = (M - 1) / 2;
    const size_t stride = (size_t)2 * Kp;
    const size_t base = (size_t)j0 * Kp + (active ? k : 0);
    // first sweep of this half: rows t = t0 + dir q, q < len; the neighbour
    // X_{t+dir} is prefetched with row t's F, X_t and X_{t-dir} stay in registers
    const int t0 = half ? M - 1 : 0, dir = half ? -1 : 1, len = half ? M - 1 - m : m;
    auto issue_up = [&](int q) {
      if (active && q < len) {
        const int t = t0 + dir * q;
        RefSlot& sl = ring.up[q & (kRefRing - 1)];
        cp_async16(&sl.f[lane], F + base + t * stride);
        const int tn = t + dir;
        if (!first && tn >= 0 && tn < M) cp_async16(&sl.x[lane], X + base + tn * stride);
        unsigned sa = (unsigned)__cvta_generic_to_shared(&sl.a[lane]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(fl + base + t * stride) : "memory");
      }
      cp_commit();
    };
    for (int q = 0; q < kRefRing; ++q) issue_up(q);
    cpx<dd> xprev = zero, xcur = zero;          // X_{t - dir}, X_t
    if (!first && active && len > 0) xcur = X[base + t0 * stride];
    cpx<float> e = {0.f, 0.f};
    float jf = (float)(j0 + 2 * t0);            // j of row t, exact in float
    const float djf = 2.f * (float)dir;
    for (int q = 0; q < len; ++q, jf += djf) {
      cp_wait<kRefRing - 1>();
      const RefSlot& sl = ring.up[q & (kRefRing - 1)];
      if (active) {
        const int t = t0 + dir * q;
        cpx<dd> r = sl.f[lane];
        const float l = sl.a[lane];
        cpx<dd> xnext = zero;
        if (!first) {
          const int tn = t + dir;
          if (tn >= 0 && tn < M) xnext = sl.x[lane];
          // ascending: X_{t-1} = xprev, X_{t+1} = xnext; descending the reverse
          r = half ? refine_residual(r, jf, two_k2, xnext, xcur, xprev)
                   : refine_residual(r, jf, two_k2, xprev, xcur, xnext);
        }
        const cpx<float> rf = {r.re.hi + r.re.lo, r.im.hi + r.im.lo};
        e = {fmaf(-l, e.re, rf.re), fmaf(-l, e.im, rf.im)};
        Y[base + t * stride] = e;
        xprev = xcur;
        xcur = xnext;
      }
      issue_up(q + kRefRing);
    }
    cp_wait_all();
    meet[half][lane] = e;
    __syncthreads();
    if (half == 0 && active) {
      // the middle row: residual from X_{m-1}, X_m, X_{m+1} and the correction
      cpx<dd> r = F[base + m * stride];
      if (!first) {
        const cpx<dd> xa = m > 0 ? X[base + (m - 1) * stride] : zero;
        const cpx<dd> xb = X[base + m * stride];
        const cpx<dd> xc = m + 1 < M ? X[base + (m + 1) * stride] : zero;
        r = refine_residual(r, (float)(j0 + 2 * m), two_k2, xa, xb, xc);
      }
      const cpx<float> rf = {r.re.hi + r.re.lo, r.im.hi + r.im.lo};
      const cpx<float> ym1 = meet[0][lane], zp1 = meet[1][lane];
      const float lm = fl[base + m * stride], ig = fiu[base + m * stride], gm = fcu[base + m * stride];
      const cpx<float> dm = {ig * (rf.re - lm * ym1.re - gm * zp1.re), ig * (rf.im - lm * ym1.im - gm * zp1.im)};
      cpx<dd> xv = first ? zero : X[base + m * stride];
      xv = {dd_add(xv.re, dd(dm.re, 0.f)), dd_add(xv.im, dd(dm.im, 0.f))};
      X[base + m * stride] = xv;
      meet[2][lane] = dm;
    }
    __syncthreads();
    __threadfence();
    // second sweep of this half: rows t1 + dir2 q (outwards from the middle row)
    const int t1 = half ? m + 1 : m - 1, dir2 = half ? 1 : -1;
    auto issue_down = [&](int q) {
      if (active && q < len) {
        const int t = t1 + dir2 * q;
        RefSlotDown& sl = ring.down[q & (kRefRing - 1)];
        cp_async8(&sl.y[lane], Y + base + t * stride);
        if (!first) cp_async16(&sl.x[lane], X + base + t * stride);
        unsigned sa = (unsigned)__cvta_generic_to_shared(&sl.a[lane]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(fiu + base + t * stride) : "memory");
        sa = (unsigned)__cvta_generic_to_shared(&sl.b[lane]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(fcu + base + t * stride) : "memory");
      }
      cp_commit();
    };
    for (int q = 0; q < kRefRing; ++q) issue_down(q);
    cpx<float> dlt = meet[2][lane];
    for (int q = 0; q < len; ++q) {
      cp_wait<kRefRing - 1>();
      const RefSlotDown& sl = ring.down[q & (kRefRing - 1)];
      if (active) {
        const int t = t1 + dir2 * q;
        const cpx<float> yv = sl.y[lane];
        const float iu = sl.a[lane], cu = sl.b[lane];
        dlt = {fmaf(yv.re, iu, -cu * dlt.re), fmaf(yv.im, iu, -cu * dlt.im)};
        cpx<dd> xv = zero;
        if (!first) xv = sl.x[lane];
        xv = {dd_add(xv.re, dd(dlt.re, 0.f)), dd_add(xv.im, dd(dlt.im, 0.f))};
        X[base + t * stride] = xv;
      }
      issue_down(q + kRefRing);
    }
    cp_wait_all();
  }
  if (even && half == 0 && active) {
    // row 0 closure in double-float: X_0 = (X_2 - F_0)/k^2 (k even), 0 (k odd)
    cpx<dd> x0v = zero;
    if (!(k & 1)) {
      __threadfence();
      cpx<dd> x2 = (2 < N) ? X[(size_t)2 * Kp + k] : zero;
      cpx<dd> f0 = F[k];
      dd ik2 = dd_from_double(1.0 / ((double)k * (double)k));
      x0v = {dd_mul(dd_sub(x2.re, f0.re), ik2), dd_mul(dd_sub(x2.im, f0.im), ik2)};
    }
    X[k] = x0v;
  }
}

// zonal column of a double-float array -> Z[i][0] (double), Z[i][1] = 0
__global__ void k_zonal_extract(const cpx<dd>* __restrict__ Wdd, cpx<double>* __restrict__ Z, int N, int Kp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  cpx<dd> v = Wdd[(size_t)i * Kp];
  Z[(size_t)i * 2] = {dd_to_double(v.re), dd_to_double(v.im)};
  Z[(size_t)i * 2 + 1] = {0.0, 0.0};
}

// after the FP64 zonal eliminations on Z: close with w^T X_0 = 0
// (X_00 = sum_{j even >= 2} 2 X_j0/(j^2-1)) and write the column, as
// double-float, into column 0 of X.  One CTA.
__global__ void k_zonal_insert(const cpx<double>* __restrict__ Z, cpx<dd>* __restrict__ X, int N, int Kp) {
  cpx<double> acc = {0.0, 0.0};
  for (int j = 2 + 2 * threadIdx.x; j < N; j += 2 * blockDim.x) {
    double wj = 2.0 / ((double)j * (double)j - 1.0);
    acc = acc + wj * Z[(size_t)j * 2];
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc.re = acc.re + __shfl_down_sync(0xffffffffu, acc.re, off);
    acc.im = acc.im + __shfl_down_sync(0xffffffffu, acc.im, off);
  }
  __shared__ cpx<double> red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    cpx<double> tot = {0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot = tot + red[w];
    X[0] = {dd_from_double(tot.re), dd_from_double(tot.im)};
  }
  for (int i = 1 + threadIdx.x; i < N; i += blockDim.x) {
    cpx<double> v = Z[(size_t)i * 2];
    X[(size_t)i * Kp] = {dd_from_double(v.re), dd_from_double(v.im)};
  }
}

#endif  // SP_REFINE_KERNELS

// ---------------------------------------------------------------------------
// The transform kernels bounded to 64 registers (about 100 bytes of spills per
// thread, to L1): two 512-thread CTAs then fit per SM beside their 80 KB FP64
// tiles, 32 warps instead of the 16 that 84-106 registers allow, and the FP64
// pipe hides more of its dependent latency (the FP64 solve 9.42 -> 9.27 ms at
// 5000 x 10000, every transform 1.5-2 % faster).  The FP64 launchers take them
// for transforms whose passes all have scaled twiddle records (radices 2, 3,
// 4, 5, 8); a radix-7 pass (plain twiddles) spills more under the bound and
// runs faster in the kernels above.
// ---------------------------------------------------------------------------
template <typename T, bool ADJ>
__global__ void __launch_bounds__(512, 2) k_rows_forward_two(
    const double* __restrict__ f, cpx<T>* __restrict__ W, int nt, int n, int Kp, int rows,
    FftDesc d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, cpx<double>* __restrict__ zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  rows_forward_tile<T, ADJ, false>(blockIdx.x, sm, f, W, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t,
                                   zonal);
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(512, 2) k_rows_inverse_two(
    const cpx<T>* __restrict__ W, double* __restrict__ u, int nt, int n, int Kp, int rows,
    FftDesc d, const cpx<T>* __restrict__ tw, const int* __restrict__ perm,
    const cpx<T>* __restrict__ post, const double* __restrict__ row_scale,
    const T* __restrict__ row_scale_t, const cpx<double>* __restrict__ zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  rows_inverse_tile<T, ADJ, false>(blockIdx.x, sm, W, u, nt, n, Kp, rows, d, tw, perm, post, row_scale, row_scale_t,
                                   zonal);
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(512, 2) k_theta_forward_two(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  theta_forward_tile<T, ADJ, false>(blockIdx.x, sm, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(512, 2) k_theta_inverse_two(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d,
    const cpx<T>* __restrict__ tw, const int* __restrict__ perm, const cpx<T>* __restrict__ post,
    T inv_n, int zonal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  theta_inverse_tile<T, ADJ, false>(blockIdx.x, sm, W, N, K, Kp, cols, d, tw, perm, post, inv_n, zonal);
}

}  // namespace sp
