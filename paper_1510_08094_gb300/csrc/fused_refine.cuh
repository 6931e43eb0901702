// Fused colatitude stage of the FP32 + refinement form (SP_FP32_REFINE):
// per wavenumber column k >= 1 (column 0 is the FP64 zonal path's), one CTA
//   1. transforms the column forward in double-float (decimation in time and
//      the DCT/DST post-twiddle in place): F, the coefficients of eq.
//      SylvesterSphericalPoisson's right-hand side, accurate to ~2^-48;
//   2. solves the per-k system of eq. linearSystems in FP32 (F rounded to
//      float, the chunked-scan eliminations of fused.cuh): X = S32 F;
//   3. refines it `sweeps` times: R = F - M X in double-float with the exact
//      band coefficients (refine_residual), X += S32 R;
//   4. closes row 0 in double-float (X_0 = (X_2 - F_0)/k^2 for even k, 0 for
//      odd k) and transforms X back (pre-twiddle in place, decimation in
//      frequency), storing the column over its input.
// F, X and the FP32 residual live in shared memory for the whole column, so
// the spectrum crosses HBM once each way instead of the unfused path's four
// times plus three per sweep.  One CTA per SM (about 200 KB of shared memory),
// persistent over the columns, with the next column's load in flight during
// the current column's inverse transform.
#pragma once

#include "fused.cuh"
#include "tma.cuh"

namespace sp {

// rows per TMA box of a column load (16 bytes per row: one double-float complex)
constexpr int kRefineBoxRows = 256;

// bytes of one double-float column buffer: N rows rounded up to whole boxes
// (a box's rows past N land there, filled with zeros by the copy)
__host__ __device__ inline size_t refine_column_bytes(int N) {
  return (size_t)((N + kRefineBoxRows - 1) / kRefineBoxRows) * kRefineBoxRows * sizeof(cpx<dd>);
}

// dynamic shared memory of k_refine_fused: the buffers start at the first
// 128-byte boundary of the dynamic region (a TMA box's shared-memory
// destination must be 128-byte aligned), hence the extra 128 bytes
__host__ __device__ inline size_t refine_fused_smem_bytes(int N, int threads) {
  const size_t a8 = ((size_t)N * sizeof(cpx<float>) + 15) & ~(size_t)15;
  return 128 + 2 * refine_column_bytes(N) + a8 + (size_t)threads * sizeof(ScanSlot<float>);
}

__device__ __forceinline__ cpx<float> round_dd(cpx<dd> v) { return {v.re.hi + v.re.lo, v.im.hi + v.im.lo}; }

// Persistent: CTA b takes the columns k = 1 + b, 1 + b + gridDim.x, ...  The
// two double-float buffers swap roles from column to column: once the row-0
// closure has read F for the last time, the next column's raw samples (one
// 16-byte element per row, in natural order) are copied into F's buffer while
// the current solution is transformed back and stored from the other; the
// next column then scatters them (Makhoul order, digit reversal) into the
// buffer just freed by the store.  The load of every column but the CTA's
// first overlaps the arithmetic of the previous one.
// With use_tma the copy is the tensor memory accelerator's: one thread issues
// ceil(N / kRefineBoxRows) 2D boxes (16 bytes x kRefineBoxRows rows of the
// [N][Kp] spectrum, tensor map tmW) completing one mbarrier, and every thread
// waits on it with a bounded poll; if the wait gives up, status is set to
// kStatusTmaTimeout and the CTA stops (uniformly, after a second bounded wait
// for the copies still in flight).  Without use_tma, each thread issues its
// share of the rows as 16-byte cp.async copies.
template <bool BIG>
__global__ void __launch_bounds__(BIG ? 256 : 512) k_refine_fused(
    cpx<dd>* __restrict__ W, int N, int K, int Kp, FftDesc d, const cpx<dd>* __restrict__ tw,
    const int* __restrict__ perm, const cpx<dd>* __restrict__ post_s, const cpx<dd>* __restrict__ post,
    const float* __restrict__ fiu, int sweeps, const __grid_constant__ CUtensorMap tmW, int use_tma,
    int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  // the first 128-byte boundary of the dynamic region (128 spare bytes are allocated)
  unsigned char* smem_al = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const size_t a16 = refine_column_bytes(N);
  const size_t a8 = ((size_t)N * sizeof(cpx<float>) + 15) & ~(size_t)15;
  cpx<dd>* A = reinterpret_cast<cpx<dd>*>(smem_al);                     // the transform, then F
  cpx<dd>* X = reinterpret_cast<cpx<dd>*>(smem_al + a16);               // raw samples, then the solution
  cpx<float>* C = reinterpret_cast<cpx<float>*>(smem_al + 2 * a16);     // FP32 right-hand sides / corrections
  ScanSlot<float>* slot = reinterpret_cast<ScanSlot<float>*>(smem_al + 2 * a16 + a8);
  const cpx<dd> zero = {dd(0.f, 0.f), dd(0.f, 0.f)};
  int k = 1 + (int)blockIdx.x;
  if (k >= K) return;                                  // uniform over the block
  const int nbox = (N + kRefineBoxRows - 1) / kRefineBoxRows;
  // column `col` into buffer `dst`: TMA boxes (thread 0) or cp.async (all threads)
  auto load_column = [&](cpx<dd>* dst, int col) {
    if (use_tma) {
      // (dst is 128-byte aligned by construction and a16 is a multiple of 4096;
      // a misaligned destination would be a fault, so it is checked: the copy is
      // then not issued and the wait below runs out and reports)
      if (threadIdx.x == 0 && (smem_u32(dst) & 127u) == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(&bar, (unsigned)(a16));
        for (int b = 0; b < nbox; ++b) tma_load_2d(dst + b * kRefineBoxRows, &tmW, 4 * col, b * kRefineBoxRows, &bar);
      }
    } else {
      stage_theta<dd>(dst, W, col, N, Kp, 1);
    }
    cp_commit();
  };
  unsigned parity = 0;
  if (use_tma && threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  load_column(X, k);                                   // the CTA's first column

  for (; k < K; k += (int)gridDim.x) {
    if (use_tma) {
      bool ok = mbar_wait_bounded(&bar, parity, kTmaPolls);
      if (__syncthreads_or(!ok)) {
        ok = mbar_wait_bounded(&bar, parity, kTmaPolls);   // the copies still in flight
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(status, kStatusTmaTimeout);
        return;
      }
      parity ^= 1u;
    } else {
      cp_wait_all();
      __syncthreads();
    }
    // 1. forward colatitude transform in double-float, F in A
    theta_forward_load<dd>(k, A, FromStaged<cpx<dd>>{X, 1}, N, K, 1, perm);
    __syncthreads();
    fft_run<-1, BIG>(A, 1, d, tw);
    post_twiddle_inplace<dd>(A, k, 1, N, K, post_s);
    __syncthreads();
    // 2. X = S32 F (rows j >= 1; row 0 is closed at the end)
    for (int j = threadIdx.x; j < N; j += blockDim.x) C[j] = round_dd(A[j]);
    __syncthreads();
    fused_solve<float>(C, 1, N, slot, k, 1, N, K, fiu);
    for (int j = threadIdx.x; j < N; j += blockDim.x)
      X[j] = j == 0 ? zero : cpx<dd>{dd(C[j].re, 0.f), dd(C[j].im, 0.f)};
    __syncthreads();
    // 3. sweeps: R = F - M X (double-float), X += S32 R
    const float kf = (float)k;
    const dd two_k2 = dd_mul(dd_prod(kf, kf), dd(2.f, 0.f));   // 2 k^2, exact
    for (int s = 0; s < sweeps; ++s) {
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        if (j == 0) {
          C[0] = {0.f, 0.f};
          continue;
        }
        const cpx<dd> xm = j >= 3 ? X[j - 2] : zero;     // rows 1 and 2 have no X_{j-2} term (a_j = 0)
        const cpx<dd> xp = j + 2 < N ? X[j + 2] : zero;
        C[j] = round_dd(refine_residual(A[j], (float)j, two_k2, xm, X[j], xp));
      }
      __syncthreads();
      fused_solve<float>(C, 1, N, slot, k, 1, N, K, fiu);
      for (int j = 1 + threadIdx.x; j < N; j += blockDim.x)
        X[j] = {dd_add(X[j].re, dd(C[j].re, 0.f)), dd_add(X[j].im, dd(C[j].im, 0.f))};
      __syncthreads();
    }
    // 4. row 0 in double-float; after it F is not read again, and A takes the
    //    next column's raw samples while X is transformed back and stored
    if (threadIdx.x == 0) {
      cpx<dd> x0 = zero;
      if (!(k & 1)) {
        const cpx<dd> x2 = N > 2 ? X[2] : zero;
        const dd ik2 = dd_from_double(1.0 / ((double)k * (double)k));
        x0 = {dd_mul(dd_sub(x2.re, A[0].re), ik2), dd_mul(dd_sub(x2.im, A[0].im), ik2)};
      }
      X[0] = x0;
    }
    __syncthreads();
    if (k + (int)gridDim.x < K) load_column(A, k + (int)gridDim.x);
    pre_twiddle_inplace<dd>(X, k, 1, N, K, post);
    __syncthreads();
    fft_run_dif<+1, BIG>(X, 1, d, tw);
    store_dif_columns<dd>(X, W, k, 1, N, K, Kp, perm);
    cpx<dd>* t = A;     // the raw samples are in A: the next column scatters them into X's buffer
    A = X;
    X = t;
  }
  cp_wait_all();
}

}  // namespace sp
