// Fused colatitude stage of the single-precision form (SP_FP32, forward solve).
//
// Per tile of `cols` consecutive wavenumber columns k, one CTA runs
//   1. the forward colatitude transform of theta_forward (the BMC fold's
//      DCT-II / DST-II, Section 4, eq. 2DFourierExpansion),
//   2. the per-k systems of eq. linearSystems on their two parity chains and
//      the j = 0 closure (as k_solve; the k = 0 column of this form is carried
//      in FP64 on the side path and replaces column 0 in rows_inverse),
//   3. the inverse colatitude transform of theta_inverse,
// with the tile's coefficients kept in shared memory between the steps: the
// spectrum crosses HBM once each way instead of three times, and the
// eliminations' factor tables are read once, column by column.
//
// The eliminations run as parallel chunked scans.  With the top-down
// factorisation of a chain (rows t = 0..M-1, j = j0 + 2t, pivots u_t; 1/u from
// k_factor_cols, stored per column so that one column's entries are
// contiguous; l_t = a_j/u_{t-1} and c_j/u_t formed from it and the closed-form
// bands a_j = (j-1)(j-2)/4, c_j = (j+1)(j+2)/4), the solve is two affine
// first-order recurrences,
//   y_t = d_t - l_t y_{t-1}           (t increasing, y_{-1} = 0),
//   x_t = (1/u_t) y_t - (c_t/u_t) x_{t+1}   (t decreasing, x_M = 0),
// each of the form z = alpha z_prev + beta.  P threads per chain take
// contiguous chunks of C rows: (1) each folds its chunk from a zero incoming
// value into (product of alpha, value at the chunk's end), (2) one warp per
// chain combines the P chunk results by a shuffle scan of the composed affine
// maps into every chunk's incoming value, (3) each thread re-runs its chunk
// from its incoming value and writes the result.  The products of alpha stay bounded (|l_t|, |c_t/u_t| < 1 on
// these diagonally dominant bands), so the scan is as accurate as the
// sequential sweep up to rounding order.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"
#include "tma.cuh"

namespace sp {

// Plan-time top-down factorisation of every parity chain, stored per column:
// entry (k, j) at k N + j of fiu holds 1/u_t for the chain row j = j0 + 2t
// (u_0 = b_j0, u_t = b_j - a_j c_{j-2} / u_{t-1}), in FP64 then rounded.
// One thread per (k, parity); idx < K the odd chain of k = idx, else the even
// chain of k = idx - K.  Rows j = 0 are not written.
template <typename S>
__global__ void k_factor_cols(S* __restrict__ fiu, int N, int K) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * K) return;
  const bool even = idx >= K;
  const int k = even ? idx - K : idx;
  const double k2 = (double)k * (double)k;
  const size_t col = (size_t)k * N;
  double u_prev = 0.0, c_prev = 0.0;
  for (int j = even ? 2 : 1, t = 0; j < N; j += 2, ++t) {
    const double jd = (double)j;
    const double a = chain_a(jd), b = -(jd * jd * 0.5 + k2), c = chain_c(jd);
    double l = 0.0, uu = b;
    if (t > 0) {
      l = a / u_prev;
      uu = b - l * c_prev;
    }
    fiu[col + j] = (S)(1.0 / uu);
    u_prev = uu;
    c_prev = c;
  }
}

// the bands of a chain row j in the arithmetic T (exact integers before the scaling)
template <typename T>
__device__ __forceinline__ T band_a(int j) { return (T)((j - 1) * (j - 2)) * (T)0.25; }
template <typename T>
__device__ __forceinline__ T band_c(int j) { return (T)((j + 1) * (j + 2)) * (T)0.25; }

// Scratch of the scans: one (product, value) pair per thread.
template <typename T>
struct ScanSlot {
  T a;
  cpx<T> z;
};

// Shared-memory bytes of the fused kernel for a tile of `cols` columns of
// length N with `threads` threads: transform buffer, coefficient buffer
// (`buffers` = 2; the single-buffer form has none), scan slots.
template <typename T>
__host__ __device__ inline size_t fused_smem_bytes(int N, int cols, int threads, int buffers = 2) {
  const size_t buf = ((size_t)cols * N * sizeof(cpx<T>) + 15) & ~(size_t)15;
  return buffers * buf + (size_t)threads * sizeof(ScanSlot<T>);
}

// The single-buffer FP32 form with two columns per CTA can take its tile by
// TMA: boxes of 16 bytes (the two columns' elements of a row) x kFusedBoxRows
// rows land in row order in the buffer (padded to whole boxes), and each thread
// then moves its kFusedTmaRegs or fewer elements through registers to their
// digit-reversed positions.
constexpr int kFusedBoxRows = 256;
constexpr int kFusedTmaRegs = 24;
__host__ __device__ inline bool fused1_tma_fits(int N, int cols, int threads) {
  return cols == 2 && threads > 0 && (2 * N + threads - 1) / threads <= kFusedTmaRegs;
}
// dynamic shared memory of the single-buffer form: the buffer (or the padded
// landing area of the TMA boxes, if larger) from a 128-byte boundary, the slots
__host__ __device__ inline size_t fused1_smem_bytes(int N, int cols, int threads) {
  const size_t buf = ((size_t)cols * N * sizeof(cpx<float>) + 15) & ~(size_t)15;
  const size_t land = (size_t)((N + kFusedBoxRows - 1) / kFusedBoxRows) * kFusedBoxRows * cols * sizeof(cpx<float>);
  return 128 + (buf > land ? buf : land) + (size_t)threads * sizeof(ScanSlot<float>);
}

// Phase 2 of one chain's scan, run by one warp: slots slot[q * stride] for the
// chunks q = 0..P-1 hold (product of alpha, value at the chunk's end from a zero
// incoming value); on return each holds the chunk's incoming value instead
// (chunks taken in increasing q, or in decreasing q when `down`).  Each lane
// folds a run of consecutive chunks, the lanes' runs are combined by a
// shuffle scan of the composed affine maps, and each lane writes its chunks'
// incoming values.
template <typename T>
__device__ __forceinline__ void chain_carry_scan(ScanSlot<T>* slot, int stride, int P, bool down) {
  const int lane = threadIdx.x & 31;
  const int Q = (P + 31) / 32;
  auto at = [&](int i) -> ScanSlot<T>& { return slot[(down ? P - 1 - i : i) * stride]; };
  // the lane's run i = lane Q .. lane Q + Q - 1 as one map z -> A z + Z
  T A = (T)1;
  cpx<T> Z = {(T)0, (T)0};
  for (int i = lane * Q; i < min(P, lane * Q + Q); ++i) {
    const ScanSlot<T> v = at(i);
    Z = {fma(v.a, Z.re, v.z.re), fma(v.a, Z.im, v.z.im)};
    A = A * v.a;
  }
  // inclusive scan over lanes: the maps of lanes 0..lane composed
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T Ao = __shfl_up_sync(0xffffffffu, A, off);
    const T Zr = __shfl_up_sync(0xffffffffu, Z.re, off);
    const T Zi = __shfl_up_sync(0xffffffffu, Z.im, off);
    if (lane >= off) {
      Z = {fma(A, Zr, Z.re), fma(A, Zi, Z.im)};
      A = A * Ao;
    }
  }
  // incoming value of the lane's run: the composed map of the lanes before it, applied to 0
  cpx<T> carry = {__shfl_up_sync(0xffffffffu, Z.re, 1), __shfl_up_sync(0xffffffffu, Z.im, 1)};
  if (lane == 0) carry = {(T)0, (T)0};
  for (int i = lane * Q; i < min(P, lane * Q + Q); ++i) {
    ScanSlot<T>& v = at(i);
    const cpx<T> out = {fma(v.a, carry.re, v.z.re), fma(v.a, carry.im, v.z.im)};
    v.z = carry;
    carry = out;
  }
}

// The eliminations of a tile and its row-0 closure, in place in X (the
// forward transform's output; coefficient (j, column c) at X[j js + c cs]), by
// the chunked scans described above.  Whole CTA; ends with a barrier.
// A thread's chunk of C rows needs the pivots 1/u_{s-1} .. 1/u_{e-1}: l_t on
// the way down, 1/u_t on the way up.  When C + 1 <= 24 they are read from the
// table once, into R registers (R = 12, 18 or 24, the smallest that holds
// them: the passes are unrolled R - 1 times), before the first scan; the four
// scan passes would otherwise each read them again.  Longer chunks read the
// table in every pass.
template <typename T, int R>
__device__ __forceinline__ void fused_solve_reg(cpx<T>* __restrict__ X, int js, int cs,
                                                ScanSlot<T>* __restrict__ slot, int k0, int cols, int N, int K,
                                                const T* __restrict__ fiu);

template <typename T>
__device__ __forceinline__ void fused_solve(cpx<T>* __restrict__ X, int js, int cs,
                                            ScanSlot<T>* __restrict__ slot, int k0, int cols, int N, int K,
                                            const T* __restrict__ fiu) {
  // thread -> (chain ch, chunk p); chain ch = column ch >> 1,
  //    parity ch & 1 (0: odd rows j = 1, 3, ..; 1: even rows j = 2, 4, ..)
  const int chains = 2 * cols;
  const int ch = threadIdx.x % chains, p = threadIdx.x / chains;
  const int P = blockDim.x / chains;
  const int c = ch >> 1, j0 = (ch & 1) ? 2 : 1;
  const int k = k0 + c;
  const int M = (j0 < N) ? (N - 1 - j0) / 2 + 1 : 0;
  const int C = ((M + P - 1) / P) | 1;        // odd, so that the chunks' rows spread over the banks
  // (C is the same for both parities: M differs by at most one row, and the rounding to odd absorbs it)
  {
    const int M1 = (1 < N) ? (N - 2) / 2 + 1 : 0;
    const int C1 = ((M1 + P - 1) / P) | 1;
    if (C1 + 1 <= 12) return fused_solve_reg<T, 12>(X, js, cs, slot, k0, cols, N, K, fiu);
    if (C1 + 1 <= 18) return fused_solve_reg<T, 18>(X, js, cs, slot, k0, cols, N, K, fiu);
    if (C1 + 1 <= 24) return fused_solve_reg<T, 24>(X, js, cs, slot, k0, cols, N, K, fiu);
  }
  const int s = min(M, p * C), e = min(M, s + C);
  const bool live = k < K && p < P;
  const size_t tcol = (size_t)(live ? k : 0) * N;
  ScanSlot<T>* mine = slot + threadIdx.x;
  // forward sweep y_t = d_t - l_t y_{t-1}, phase 1
  {
    T A = (T)1;
    cpx<T> y = {(T)0, (T)0};
    if (live) {
#pragma unroll 4
      for (int t = s; t < e; ++t) {
        const int j = j0 + 2 * t;
        const T l = t > 0 ? band_a<T>(j) * __ldg(fiu + tcol + j - 2) : (T)0;
        const cpx<T> dv = X[j * js + c * cs];
        y = {fma(-l, y.re, dv.re), fma(-l, y.im, dv.im)};
        A = A * (-l);
      }
    }
    mine->a = A;
    mine->z = y;
  }
  __syncthreads();
  // phase 2: chunk p's incoming value, in its slot (warp w scans chain w)
  {
    const int w = threadIdx.x >> 5;
    if (w < chains && k0 + (w >> 1) < K) chain_carry_scan(slot + w, chains, P, false);
  }
  __syncthreads();
  // phase 3
  if (live) {
    cpx<T> y = mine->z;
    for (int t = s; t < e; ++t) {
      const int j = j0 + 2 * t;
      const T l = t > 0 ? band_a<T>(j) * __ldg(fiu + tcol + j - 2) : (T)0;
      cpx<T>& dv = X[j * js + c * cs];
      y = {fma(-l, y.re, dv.re), fma(-l, y.im, dv.im)};
      dv = y;
    }
  }
  __syncthreads();
  // backward sweep x_t = iu_t y_t - cu_t x_{t+1} (t decreasing), phase 1
  {
    T A = (T)1;
    cpx<T> x = {(T)0, (T)0};
    if (live) {
#pragma unroll 4
      for (int t = e - 1; t >= s; --t) {
        const int j = j0 + 2 * t;
        const T iu = __ldg(fiu + tcol + j), cu = band_c<T>(j) * iu;
        const cpx<T> yv = X[j * js + c * cs];
        x = {fma(iu, yv.re, -cu * x.re), fma(iu, yv.im, -cu * x.im)};
        A = A * (-cu);
      }
    }
    mine->a = A;
    mine->z = x;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5;
    if (w < chains && k0 + (w >> 1) < K) chain_carry_scan(slot + w, chains, P, true);
  }
  __syncthreads();
  if (live) {
    cpx<T> x = mine->z;
    for (int t = e - 1; t >= s; --t) {
      const int j = j0 + 2 * t;
      const T iu = __ldg(fiu + tcol + j), cu = band_c<T>(j) * iu;
      cpx<T>& yv = X[j * js + c * cs];
      x = {fma(iu, yv.re, -cu * x.re), fma(iu, yv.im, -cu * x.im)};
      yv = x;
    }
  }
  __syncthreads();
  // row 0: k even != 0: X_0 = (X_2 - F_0)/k^2 (row 0 with X_{-2,k} = X_{2,k});
  // k odd: X_0 = 0; k = 0: left to the FP64 zonal column
  if (threadIdx.x < cols) {
    const int kc = k0 + threadIdx.x;
    if (kc < K && kc != 0) {
      cpx<T>& x0 = X[threadIdx.x * cs];
      if (kc & 1) {
        x0 = {(T)0, (T)0};
      } else {
        const T ik2 = (T)(1.0 / ((double)kc * (double)kc));
        const cpx<T> x2 = N > 2 ? X[2 * js + threadIdx.x * cs] : cpx<T>{(T)0, (T)0};
        x0 = {(x2.re - x0.re) * ik2, (x2.im - x0.im) * ik2};
      }
    }
  }
  __syncthreads();
}

// fused_solve with the chunk's pivots in registers (C + 1 <= R): the same
// scans, passes and row-0 closure.  Whole CTA; ends with a barrier.
template <typename T, int R>
__device__ __forceinline__ void fused_solve_reg(cpx<T>* __restrict__ X, int js, int cs,
                                                ScanSlot<T>* __restrict__ slot, int k0, int cols, int N, int K,
                                                const T* __restrict__ fiu) {
  const int chains = 2 * cols;
  const int ch = threadIdx.x % chains, p = threadIdx.x / chains;
  const int P = blockDim.x / chains;
  const int c = ch >> 1, j0 = (ch & 1) ? 2 : 1;
  const int k = k0 + c;
  const int M = (j0 < N) ? (N - 1 - j0) / 2 + 1 : 0;
  const int C = ((M + P - 1) / P) | 1;
  const int s = min(M, p * C), e = min(M, s + C);
  const bool live = k < K && p < P;
  const size_t tcol = (size_t)(live ? k : 0) * N;
  ScanSlot<T>* mine = slot + threadIdx.x;
  cpx<T>* Xc = X + c * cs;
  // iu[q] = 1/u_{s-1+q} for q = 0 .. e - s (zero where t < 0 or past the chunk)
  T iu[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int t = s - 1 + q;
    iu[q] = (live && t >= 0 && t < e) ? __ldg(fiu + tcol + j0 + 2 * t) : (T)0;
  }
  // forward sweep y_t = d_t - l_t y_{t-1}, l_t = a_j / u_{t-1} (l_0 = 0 since iu[0] = 0 at s = 0)
  {
    T A = (T)1;
    cpx<T> y = {(T)0, (T)0};
#pragma unroll
    for (int q = 0; q < R - 1; ++q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T l = band_a<T>(j) * iu[q];
        const cpx<T> dv = Xc[j * js];
        y = {fma(-l, y.re, dv.re), fma(-l, y.im, dv.im)};
        A = A * (-l);
      }
    }
    mine->a = A;
    mine->z = y;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5;
    if (w < chains && k0 + (w >> 1) < K) chain_carry_scan(slot + w, chains, P, false);
  }
  __syncthreads();
  {
    cpx<T> y = mine->z;
#pragma unroll
    for (int q = 0; q < R - 1; ++q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T l = band_a<T>(j) * iu[q];
        cpx<T>& dv = Xc[j * js];
        y = {fma(-l, y.re, dv.re), fma(-l, y.im, dv.im)};
        dv = y;
      }
    }
  }
  __syncthreads();
  // backward sweep x_t = iu_t y_t - cu_t x_{t+1} (t decreasing), iu_t = iu[t - s + 1]
  {
    T A = (T)1;
    cpx<T> x = {(T)0, (T)0};
#pragma unroll
    for (int q = R - 2; q >= 0; --q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T u = iu[q + 1], cu = band_c<T>(j) * u;
        const cpx<T> yv = Xc[j * js];
        x = {fma(u, yv.re, -cu * x.re), fma(u, yv.im, -cu * x.im)};
        A = A * (-cu);
      }
    }
    mine->a = A;
    mine->z = x;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5;
    if (w < chains && k0 + (w >> 1) < K) chain_carry_scan(slot + w, chains, P, true);
  }
  __syncthreads();
  {
    cpx<T> x = mine->z;
#pragma unroll
    for (int q = R - 2; q >= 0; --q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T u = iu[q + 1], cu = band_c<T>(j) * u;
        cpx<T>& yv = Xc[j * js];
        x = {fma(u, yv.re, -cu * x.re), fma(u, yv.im, -cu * x.im)};
        yv = x;
      }
    }
  }
  __syncthreads();
  // row 0 as in fused_solve
  if (threadIdx.x < cols) {
    const int kc = k0 + threadIdx.x;
    if (kc < K && kc != 0) {
      cpx<T>& x0 = X[threadIdx.x * cs];
      if (kc & 1) {
        x0 = {(T)0, (T)0};
      } else {
        const T ik2 = (T)(1.0 / ((double)kc * (double)kc));
        const cpx<T> x2 = N > 2 ? X[2 * js + threadIdx.x * cs] : cpx<T>{(T)0, (T)0};
        x0 = {(x2.re - x0.re) * ik2, (x2.im - x0.im) * ik2};
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The transposed eliminations of the adjoint (the transpose of fused_solve):
// with the same top-down factorisation M = L U of each chain,
//   U^T p = b:  p_t = (1/u_t) (b_t - c_{j-2} p_{t-1})          (t increasing),
//   L^T r = p:  r_t = p_t - (a_{j+2}/u_t) r_{t+1}               (t decreasing),
// both affine first-order recurrences run as the same chunked scans, and before
// them the transposed row-0 closure: for even k != 0, Fbar_0 = -Xbar_0/k^2 and
// Xbar_2 += Xbar_0/k^2; for odd k and k = 0, Fbar_0 = 0 (the k = 0 column is the
// FP64 zonal path's).  Pivots from the per-column table, in registers when the chunk is
// short enough (R of them), else read in each pass.  Whole CTA; ends with a
// barrier.
template <typename T, int R>
__device__ __forceinline__ void fused_solve_adj_impl(cpx<T>* __restrict__ X, int js, int cs,
                                                     ScanSlot<T>* __restrict__ slot, int k0, int cols, int N,
                                                     int K, const T* __restrict__ fiu) {
  // transposed closure of row 0, then the chains on rows j >= 1
  if (threadIdx.x < cols) {
    const int kc = k0 + threadIdx.x;
    if (kc < K) {
      cpx<T>& x0 = X[threadIdx.x * cs];
      const cpx<T> xb0 = x0;
      if (kc == 0 || (kc & 1)) {
        x0 = {(T)0, (T)0};
      } else {
        const T ik2 = (T)(1.0 / ((double)kc * (double)kc));
        x0 = {-xb0.re * ik2, -xb0.im * ik2};
        if (N > 2) {
          cpx<T>& x2 = X[2 * js + threadIdx.x * cs];
          x2 = {fma(ik2, xb0.re, x2.re), fma(ik2, xb0.im, x2.im)};
        }
      }
    }
  }
  __syncthreads();
  const int chains = 2 * cols;
  const int ch = threadIdx.x % chains, p = threadIdx.x / chains;
  const int P = blockDim.x / chains;
  const int c = ch >> 1, j0 = (ch & 1) ? 2 : 1;
  const int k = k0 + c;
  const int M = (j0 < N) ? (N - 1 - j0) / 2 + 1 : 0;
  const int C = ((M + P - 1) / P) | 1;
  const int s = min(M, p * C), e = min(M, s + C);
  const bool live = k < K && p < P;
  const size_t tcol = (size_t)(live ? k : 0) * N;
  ScanSlot<T>* mine = slot + threadIdx.x;
  cpx<T>* Xc = X + c * cs;
  // pivot of chain row t (t in the chunk)
  T iu[R > 0 ? R : 1];
  if constexpr (R > 0) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int t = s + q;
      iu[q] = (live && t < e) ? __ldg(fiu + tcol + j0 + 2 * t) : (T)0;
    }
  }
  auto piv = [&](int q, int t) -> T {
    if constexpr (R > 0) return iu[q];
    else return __ldg(fiu + tcol + j0 + 2 * t);
  };
  const int span = R > 0 ? R : C;     // loop bound (rows past e are skipped)
  // U^T p = b: p_t = iu_t b_t - (c_{j-2} iu_t) p_{t-1}
  {
    T A = (T)1;
    cpx<T> z = {(T)0, (T)0};
#pragma unroll
    for (int q = 0; q < span; ++q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T u = piv(q, t);
        const T al = t > 0 ? -band_c<T>(j - 2) * u : (T)0;
        const cpx<T> b = Xc[j * js];
        z = {fma(al, z.re, u * b.re), fma(al, z.im, u * b.im)};
        A = A * al;
      }
    }
    mine->a = A;
    mine->z = z;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5;
    if (w < chains && k0 + (w >> 1) < K) chain_carry_scan(slot + w, chains, P, false);
  }
  __syncthreads();
  {
    cpx<T> z = mine->z;
#pragma unroll
    for (int q = 0; q < span; ++q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T u = piv(q, t);
        const T al = t > 0 ? -band_c<T>(j - 2) * u : (T)0;
        cpx<T>& b = Xc[j * js];
        z = {fma(al, z.re, u * b.re), fma(al, z.im, u * b.im)};
        b = z;
      }
    }
  }
  __syncthreads();
  // L^T r = p: r_t = p_t - (a_{j+2} iu_t) r_{t+1}
  {
    T A = (T)1;
    cpx<T> z = {(T)0, (T)0};
#pragma unroll
    for (int q = span - 1; q >= 0; --q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T al = t < M - 1 ? -band_a<T>(j + 2) * piv(q, t) : (T)0;
        const cpx<T> pv = Xc[j * js];
        z = {fma(al, z.re, pv.re), fma(al, z.im, pv.im)};
        A = A * al;
      }
    }
    mine->a = A;
    mine->z = z;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5;
    if (w < chains && k0 + (w >> 1) < K) chain_carry_scan(slot + w, chains, P, true);
  }
  __syncthreads();
  {
    cpx<T> z = mine->z;
#pragma unroll
    for (int q = span - 1; q >= 0; --q) {
      const int t = s + q;
      if (live && t < e) {
        const int j = j0 + 2 * t;
        const T al = t < M - 1 ? -band_a<T>(j + 2) * piv(q, t) : (T)0;
        cpx<T>& pv = Xc[j * js];
        z = {fma(al, z.re, pv.re), fma(al, z.im, pv.im)};
        pv = z;
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void fused_solve_adj(cpx<T>* __restrict__ X, int js, int cs,
                                                ScanSlot<T>* __restrict__ slot, int k0, int cols, int N, int K,
                                                const T* __restrict__ fiu) {
  const int P = blockDim.x / (2 * cols);
  const int M1 = (1 < N) ? (N - 2) / 2 + 1 : 0;
  const int C1 = ((M1 + P - 1) / P) | 1;
  if (C1 <= 12) return fused_solve_adj_impl<T, 12>(X, js, cs, slot, k0, cols, N, K, fiu);
  if (C1 <= 18) return fused_solve_adj_impl<T, 18>(X, js, cs, slot, k0, cols, N, K, fiu);
  if (C1 <= 24) return fused_solve_adj_impl<T, 24>(X, js, cs, slot, k0, cols, N, K, fiu);
  fused_solve_adj_impl<T, 0>(X, js, cs, slot, k0, cols, N, K, fiu);
}

template <typename T, bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_theta_fused(
    cpx<T>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d, const cpx<T>* __restrict__ tw,
    const int* __restrict__ perm, const cpx<T>* __restrict__ post_s, const cpx<T>* __restrict__ post,
    const T* __restrict__ fiu, T inv_n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t buf = ((size_t)cols * N * sizeof(cpx<T>) + 15) & ~(size_t)15;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);                 // FFT buffer, [c][N] permuted
  cpx<T>* X = reinterpret_cast<cpx<T>*>(smem_raw + buf);            // coefficients, [j][cols]
  ScanSlot<T>* slot = reinterpret_cast<ScanSlot<T>*>(smem_raw + 2 * buf);
  const int k0 = blockIdx.x * cols;

  // 1. forward colatitude transform into X (theta_forward with the tile's
  //    coefficient buffer as its output array: row stride cols, column k - k0)
  theta_forward_load<T>(k0, sm, FromGlobal<cpx<T>>{W + k0, (size_t)Kp}, N, K, cols, perm);
  __syncthreads();
  theta_forward_finish<T, false, BIG>(k0, sm, X - k0, N, K, cols, cols, d, tw, post_s, 0);
  __syncthreads();

  // 2. eliminations and the row-0 closure, in X
  fused_solve<T>(X, cols, 1, slot, k0, cols, N, K, fiu);

  // 3. inverse colatitude transform from X back to W
  theta_inverse_load<T, false>(k0, sm, FromStaged<cpx<T>>{X, cols}, N, K, cols, perm, post, 0);
  __syncthreads();
  theta_inverse_finish<T, false, BIG>(k0, sm, W, N, K, Kp, cols, d, tw, inv_n);
}

// Cluster form: a cluster of kFuseCluster = 4 CTAs takes four consecutive
// columns, one per CTA, and the CTAs share the tile's global traffic through
// distributed shared memory: CTA r loads (and at the end stores) every fourth
// row of all four columns, 32 contiguous bytes per row, and scatters the
// values into (gathers them from) the four CTAs' transform buffers.  A column
// of this layout alone is 8 scattered bytes per row, a quarter of a 32-byte
// sector; four neighbouring columns fill the sector.  FP32 arithmetic only
// (one complex value = 8 bytes, four = two 16-byte vectors).
constexpr int kFuseCluster = 4;

template <bool BIG>
__global__ void __cluster_dims__(kFuseCluster, 1, 1) __launch_bounds__(BIG ? 256 : 512) k_theta_fused_cl(
    cpx<float>* __restrict__ W, int N, int K, int Kp, FftDesc d, const cpx<float>* __restrict__ tw,
    const int* __restrict__ perm, const cpx<float>* __restrict__ post_s, const cpx<float>* __restrict__ post,
    const float* __restrict__ fiu) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int kc0 = (int)(blockIdx.x / kFuseCluster) * kFuseCluster;   // the cluster's first column
  const int k = kc0 + r;                                              // this CTA's column
  const size_t buf = ((size_t)N * sizeof(cpx<float>) + 15) & ~(size_t)15;
  cpx<float>* sm = reinterpret_cast<cpx<float>*>(smem_raw);          // this column's transform buffer
  cpx<float>* X = reinterpret_cast<cpx<float>*>(smem_raw + buf);     // its coefficients
  ScanSlot<float>* slot = reinterpret_cast<ScanSlot<float>*>(smem_raw + 2 * buf);
  cpx<float>* peer[kFuseCluster];
#pragma unroll
  for (int q = 0; q < kFuseCluster; ++q) peer[q] = cluster.map_shared_rank(sm, q);
  // the two 16-byte halves of a row's four columns exist when their first column is
  // below Kp (Kp is even and kc0 a multiple of 4, so the second column is too)
  const bool half1 = kc0 + 2 < Kp;

  // 1. load: rows i = r, r + 4, ..; the Makhoul reordering with (-1)^i on odd k and
  //    the digit-reversed position as in theta_forward_load
  for (int i = r + kFuseCluster * (int)threadIdx.x; i < N; i += kFuseCluster * (int)blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(W + (size_t)i * Kp + kc0);
    const float4 a = src[0];
    const float4 b = half1 ? src[1] : make_float4(0.f, 0.f, 0.f, 0.f);
    const cpx<float> v[kFuseCluster] = {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}, {b.z, b.w}};
    const int pos = __ldg(perm + makhoul_pos(i, N));
#pragma unroll
    for (int q = 0; q < kFuseCluster; ++q) {
      const int kq = kc0 + q;
      peer[q][pos] = kq < K ? neg_if(v[q], (kq & 1) && (i & 1)) : cpx<float>{0.f, 0.f};
    }
  }
  cluster.sync();

  // 2. this column: forward transform into X, eliminations, inverse transform in sm
  theta_forward_finish<float, false, BIG>(k, sm, X - k, N, K, 1, 1, d, tw, post_s, 0);
  __syncthreads();
  fused_solve<float>(X, 1, 1, slot, k, 1, N, K, fiu);
  theta_inverse_load<float, false>(k, sm, FromStaged<cpx<float>>{X, 1}, N, K, 1, perm, post, 0);
  __syncthreads();
  fft_run<+1, BIG>(sm, 1, d, tw);
  cluster.sync();

  // 3. store: rows i = r, r + 4, ..; the inverse Makhoul reordering and, on odd
  //    k, the factor i (-1)^i as in theta_inverse_finish
  for (int i = r + kFuseCluster * (int)threadIdx.x; i < N; i += kFuseCluster * (int)blockDim.x) {
    const int pos = makhoul_pos(i, N);
    cpx<float> v[kFuseCluster];
#pragma unroll
    for (int q = 0; q < kFuseCluster; ++q) {
      const cpx<float> x = peer[q][pos];
      v[q] = ((kc0 + q) & 1) ? cpx<float>{neg_if(x.im, !(i & 1)), neg_if(x.re, (i & 1) != 0)} : x;
    }
    float4* dst = reinterpret_cast<float4*>(W + (size_t)i * Kp + kc0);
    dst[0] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
    if (half1) dst[1] = make_float4(v[2].re, v[2].im, v[3].re, v[3].im);
  }
  cluster.sync();   // no CTA leaves while a peer still reads its buffer
}

// In-place DCT/DST post-twiddle of the forward colatitude transform on
// natural-order pairs (j, N - j) of each column c of sm ([c][N]), the forward
// form of theta_forward_finish: each thread reads a pair and writes the same
// pair.  Columns k >= K are left alone.
// ADJ: the adjoint's form (the transpose of theta_inverse, as theta_forward's
// adjoint): called with the unscaled table, the j = 0 output of even k halved.
template <typename T, bool ADJ = false>
__device__ __forceinline__ void post_twiddle_inplace(cpx<T>* __restrict__ sm, int k0, int cols, int N, int K,
                                                     const cpx<T>* __restrict__ post_s) {
  const int cs = __ffs(cols) - 1;
  const int H = N / 2 + 1;
  for (int idx = threadIdx.x; idx < H * cols; idx += blockDim.x) {
    const int j = idx >> cs, c = idx & (cols - 1);
    const int k = k0 + c;
    if (k >= K) continue;
    cpx<T>* V = sm + c * N;
    const int jj = N - j;
    const bool pair = j > 0 && jj != j;
    const cpx<T> w = ldg_c(post_s + j);
    const cpx<T> a = V[j], b = V[j == 0 ? 0 : jj];
    const cpx<T> S = a + b, D = a - b;
    const cpx<T> pj = {fma(w.re, S.re, -(w.im * D.im)), fma(w.re, S.im, w.im * D.re)};
    const cpx<T> pjj = {fma(-w.im, S.re, -(w.re * D.im)), fma(-w.im, S.im, w.re * D.re)};
    if ((k & 1) == 0) {
      V[j] = (ADJ && j == 0) ? cpx<T>{(T)0.5 * pj.re, (T)0.5 * pj.im} : pj;
      if (pair) V[jj] = pjj;
    } else {
      V[j] = j == 0 ? cpx<T>{(T)0, (T)0} : cpx<T>{pjj.im, -pjj.re};
      if (pair) V[jj] = {pj.im, -pj.re};
    }
  }
}

// In-place pre-twiddle of the inverse colatitude transform (the forward form
// of theta_inverse_load) in natural order; columns k >= K are zeroed.
// ADJ: the adjoint's form (the transpose of theta_forward): inputs j >= 1 halved.
template <typename T, bool ADJ = false>
__device__ __forceinline__ void pre_twiddle_inplace(cpx<T>* __restrict__ sm, int k0, int cols, int N, int K,
                                                    const cpx<T>* __restrict__ post) {
  const int cs = __ffs(cols) - 1;
  const int H = N / 2 + 1;
  for (int idx = threadIdx.x; idx < H * cols; idx += blockDim.x) {
    const int j = idx >> cs, c = idx & (cols - 1);
    const int k = k0 + c;
    cpx<T>* V = sm + c * N;
    const int jj = N - j;
    const bool odd = (k & 1);
    if (k >= K) {
      V[j] = {(T)0, (T)0};
      if (j > 0 && jj != j) V[jj] = {(T)0, (T)0};
      continue;
    }
    if (j == 0) {
      if (odd) V[0] = {(T)0, (T)0};
      continue;
    }
    cpx<T> xa = V[j], xb = V[jj];
    if (ADJ) {
      xa = {(T)0.5 * xa.re, (T)0.5 * xa.im};
      xb = {(T)0.5 * xb.re, (T)0.5 * xb.im};
    }
    const cpx<T> ya = odd ? xb : xa, yb = odd ? xa : xb;
    V[j] = cmul(conj(ldg_c(post + j)), cpx<T>{ya.re + yb.im, ya.im - yb.re});
    if (jj != j) V[jj] = cmul(conj(ldg_c(post + jj)), cpx<T>{yb.re + ya.im, yb.im - ya.re});
  }
}

// The store after a decimation-in-frequency inverse: output i of column c is
// at sm[c N + perm[makhoul_pos(i, N)]]; on odd k the factor i (-1)^i; SCALED:
// times `scale` (the adjoint's 1/N).
template <typename T, bool SCALED = false>
__device__ __forceinline__ void store_dif_columns(const cpx<T>* __restrict__ sm, cpx<T>* __restrict__ W, int k0,
                                                  int cols, int N, int K, int Kp, const int* __restrict__ perm,
                                                  T scale = (T)1) {
  const int cs = __ffs(cols) - 1;
  for (int idx = threadIdx.x; idx < N * cols; idx += blockDim.x) {
    const int i = idx >> cs, c = idx & (cols - 1);
    const int k = k0 + c;
    if (k >= K) continue;
    cpx<T> v = sm[c * N + __ldg(perm + makhoul_pos(i, N))];
    if (k & 1) v = {neg_if(v.im, !(i & 1)), neg_if(v.re, (i & 1) != 0)};
    if (SCALED) v = {scale * v.re, scale * v.im};
    W[(size_t)i * Kp + k] = v;
  }
}

// The tile load of the single-buffer kernels: columns [k0, k0 + cols) of W
// (Makhoul reordering, digit-reversed positions; the factor (-1)^i on odd k)
// into sm, by TMA with use_tma (two columns per CTA) or by per-thread loads.
// false (uniformly over the block) if the TMA wait gave up; ends with a barrier.
__device__ __forceinline__ bool fused1_load(cpx<float>* sm, uint64_t& bar, const cpx<float>* __restrict__ W, int N,
                                            int K, int Kp, int cols, int k0, const int* __restrict__ perm,
                                            const CUtensorMap* tmW, int use_tma, int* __restrict__ status) {
  const int nbox = (N + kFusedBoxRows - 1) / kFusedBoxRows;
  const size_t land = (size_t)nbox * kFusedBoxRows * cols * sizeof(cpx<float>);
  if (use_tma) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      mbar_init_fence();
    }
    __syncthreads();
    // (sm is 128-byte aligned by construction and each box is 4096 bytes; a
    // misaligned destination is not issued, and the wait below reports it)
    if (threadIdx.x == 0 && (smem_u32(sm) & 127u) == 0) {
      mbar_expect_tx(&bar, (unsigned)land);
      for (int b = 0; b < nbox; ++b) tma_load_2d(sm + b * kFusedBoxRows * 2, tmW, 2 * k0, b * kFusedBoxRows, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, kTmaPolls);
    if (__syncthreads_or(!ok)) {
      mbar_wait_bounded(&bar, 0, kTmaPolls);            // the copies still in flight
      __syncthreads();
      if (threadIdx.x == 0) atomicExch(status, kStatusTmaTimeout);
      return false;
    }
    // row-ordered elements e = 2 i + c to their digit-reversed positions, through registers
    cpx<float> v[kFusedTmaRegs];
#pragma unroll
    for (int t = 0; t < kFusedTmaRegs; ++t) {
      const int e = (int)threadIdx.x + t * (int)blockDim.x;
      if (e < 2 * N) v[t] = sm[e];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kFusedTmaRegs; ++t) {
      const int e = (int)threadIdx.x + t * (int)blockDim.x;
      if (e < 2 * N) {
        const int i = e >> 1, c = e & 1, k = k0 + c;
        const cpx<float> z = k < K ? neg_if(v[t], (k & 1) && (i & 1)) : cpx<float>{0.f, 0.f};
        sm[c * N + __ldg(perm + makhoul_pos(i, N))] = z;
      }
    }
  } else {
    theta_forward_load<float>(k0, sm, FromGlobal<cpx<float>>{W + k0, (size_t)Kp}, N, K, cols, perm);
  }
  __syncthreads();
  return true;
}

// Single-buffer form: the tile lives in one shared-memory buffer ([c][N]) from
// load to store.  The forward transform runs by decimation in time (digit-
// reversed input, natural output), the DCT/DST post-twiddle, the eliminations
// and the inverse pre-twiddle work in place on natural-order pairs (j, N - j),
// and the inverse transform runs by decimation in frequency (natural input,
// digit-reversed output), read back through the same permutation at the store.
// Half the shared memory of the two-buffer form, so two columns per CTA keep
// two CTAs per SM.
//
// With use_tma (two columns per CTA, fused1_tma_fits) the tile arrives by TMA
// (tensor map tmW: the [N][Kp] spectrum as 32-bit words) on an mbarrier with a
// bounded wait; a wait that gives up sets *status = kStatusTmaTimeout and the
// CTA stops.
template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512, BIG ? 1 : 2) k_theta_fused1(
    cpx<float>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d, const cpx<float>* __restrict__ tw,
    const int* __restrict__ perm, const cpx<float>* __restrict__ post_s, const cpx<float>* __restrict__ post,
    const float* __restrict__ fiu, const __grid_constant__ CUtensorMap tmW, int use_tma,
    int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  // the first 128-byte boundary of the dynamic region (128 spare bytes are allocated)
  unsigned char* smem_al = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const size_t buf = ((size_t)cols * N * sizeof(cpx<float>) + 15) & ~(size_t)15;
  const int nbox = (N + kFusedBoxRows - 1) / kFusedBoxRows;
  const size_t land = (size_t)nbox * kFusedBoxRows * cols * sizeof(cpx<float>);
  cpx<float>* sm = reinterpret_cast<cpx<float>*>(smem_al);
  ScanSlot<float>* slot = reinterpret_cast<ScanSlot<float>*>(smem_al + (buf > land ? buf : land));
  const int k0 = blockIdx.x * cols;

  // 1. load (Makhoul reordering, digit-reversed positions) and forward DIT transform
  if (!fused1_load(sm, bar, W, N, K, Kp, cols, k0, perm, &tmW, use_tma, status)) return;
  fft_run<-1, BIG>(sm, cols, d, tw);
  // 2. post-twiddle in place on the pairs (j, N - j) (theta_forward_finish, forward form)
  post_twiddle_inplace<float>(sm, k0, cols, N, K, post_s);
  __syncthreads();
  // 3. eliminations in place
  fused_solve<float>(sm, 1, N, slot, k0, cols, N, K, fiu);
  // 4. pre-twiddle of the inverse in place (theta_inverse_load, forward form),
  //    in natural order
  pre_twiddle_inplace<float>(sm, k0, cols, N, K, post);
  __syncthreads();
  // 5. inverse DIF transform (output q at position perm[q]) and store with the
  //    inverse Makhoul reordering and, on odd k, the factor i (-1)^i
  fft_run_dif<+1, BIG>(sm, cols, d, tw);
  store_dif_columns<float>(sm, W, k0, cols, N, K, Kp, perm);
}

// The adjoint's colatitude stage in the same single buffer: the transposes of
// theta_inverse (the forward DIT transform, the post-twiddle with the unscaled
// table and the j = 0 output of even k halved), of the eliminations
// (fused_solve_adj) and of theta_forward (the pre-twiddle with inputs j >= 1
// halved, the DIF inverse, the store scaled by inv_n = 1/N): what
// theta_forward<ADJ>, k_solve<ADJ> and theta_inverse<ADJ> compute in three
// launches.
template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512, BIG ? 1 : 2) k_theta_fused1_adj(
    cpx<float>* __restrict__ W, int N, int K, int Kp, int cols, FftDesc d, const cpx<float>* __restrict__ tw,
    const int* __restrict__ perm, const cpx<float>* __restrict__ post, const float* __restrict__ fiu, float inv_n,
    const __grid_constant__ CUtensorMap tmW, int use_tma, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  unsigned char* smem_al = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const size_t buf = ((size_t)cols * N * sizeof(cpx<float>) + 15) & ~(size_t)15;
  const int nbox = (N + kFusedBoxRows - 1) / kFusedBoxRows;
  const size_t land = (size_t)nbox * kFusedBoxRows * cols * sizeof(cpx<float>);
  cpx<float>* sm = reinterpret_cast<cpx<float>*>(smem_al);
  ScanSlot<float>* slot = reinterpret_cast<ScanSlot<float>*>(smem_al + (buf > land ? buf : land));
  const int k0 = blockIdx.x * cols;

  if (!fused1_load(sm, bar, W, N, K, Kp, cols, k0, perm, &tmW, use_tma, status)) return;
  fft_run<-1, BIG>(sm, cols, d, tw);
  post_twiddle_inplace<float, true>(sm, k0, cols, N, K, post);
  __syncthreads();
  fused_solve_adj<float>(sm, 1, N, slot, k0, cols, N, K, fiu);
  pre_twiddle_inplace<float, true>(sm, k0, cols, N, K, post);
  __syncthreads();
  fft_run_dif<+1, BIG>(sm, cols, d, tw);
  store_dif_columns<float, true>(sm, W, k0, cols, N, K, Kp, perm, inv_n);
}

}  // namespace sp
