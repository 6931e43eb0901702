// FP64 operators on the coefficients and samples of one sphere, beside the
// solve: the surface integral (Section 4, Integration), the tangential
// derivatives and vector calculus (Section 4, Differentiation and vector-valued
// functions), the structure-preserving Gaussian elimination and the low-rank
// right-hand side (Section 3).  Included by the FP64 translation unit only.
#pragma once

#include "kernels.cuh"

namespace sp {

// Surface integral from the k = 0 coefficient column A_j (j >= 0) of f~
// (Section 4, Integration, eq. integrationCoeffs): int_S f = 2 pi sum_j w_j A_j
// over j = -(N-1)..N-1, w_j = 2/(1-j^2) for even j, 0 for odd j; the column is
// theta-even (A_{-j} = A_j), so the sum is 2 A_0 + 4 sum_{j even >= 2} A_j/(1-j^2).
__global__ void k_sum2_finish(const cpx<double>* __restrict__ C, int N, int Kp, double* __restrict__ out) {
  double acc = 0.0;
  for (int j = 2 + 2 * threadIdx.x; j < N; j += 2 * blockDim.x) {
    double jd = (double)j;
    acc += C[(size_t)j * Kp].re / (1.0 - jd * jd);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const double two_pi = 6.283185307179586476925286766559;
    *out = two_pi * (2.0 * C[0].re + 4.0 * t);
  }
}

// Mean of f over the sphere, (1/4 pi) int_S f, by the same quadrature as the
// surface integral above (eq. integrationCoeffs on the DFS interpolant, the
// theta-Nyquist mode dropped), written on the grid values: the lambda mean of
// row i is (1/n) sum_q f_iq, and the colatitude quadrature is the plan's row
// weight w_i, so mean = sum_i sum_q (w_i / n) f_iq with wrow[i] = w_i / n.
// Pass 1: each CTA takes rows blockIdx.x, blockIdx.x + gridDim.x, ... and
// writes (its weighted sum, the largest |f_iq| as the bits of a non-negative
// double) to part[blockIdx.x]; pass 2 (one CTA) adds the parts in a fixed
// order, so the result does not depend on scheduling.  Rows are read as
// 16-byte pairs (n even, f 16-byte aligned).  blockDim.x: a multiple of 32, <= 1024.
__device__ __forceinline__ void block_sum_max(double& s, unsigned long long& mx) {
  __shared__ double rs[32];
  __shared__ unsigned long long rm[32];
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, off);
    const unsigned long long o = __shfl_down_sync(0xffffffffu, mx, off);
    mx = o > mx ? o : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = s;
    rm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += rs[w];
      m = rm[w] > m ? rm[w] : m;
    }
    s = t;
    mx = m;
  }
}

__global__ void k_mean_partial(const double* __restrict__ f, int nt, int n, const double* __restrict__ wrow,
                               double2* __restrict__ part) {
  double acc = 0.0;
  unsigned long long mx = 0;
  const int half = n >> 1;
  for (int i = blockIdx.x; i < nt; i += gridDim.x) {
    const double2* row = reinterpret_cast<const double2*>(f + (size_t)i * n);
    double s = 0.0;
    for (int q = threadIdx.x; q < half; q += blockDim.x) {
      const double2 v = row[q];
      s += v.x + v.y;
      const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
      const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
      const unsigned long long ab = a > b ? a : b;
      mx = ab > mx ? ab : mx;
    }
    acc = fma(wrow[i], s, acc);
  }
  block_sum_max(acc, mx);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(acc, __longlong_as_double((long long)mx));
}

__global__ void k_mean_final(const double2* __restrict__ part, int nparts, double* __restrict__ mean,
                             double* __restrict__ absmax) {
  double s = 0.0;
  unsigned long long mx = 0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    const double2 v = part[b];
    s += v.x;
    const unsigned long long m = (unsigned long long)__double_as_longlong(v.y);
    mx = m > mx ? m : mx;
  }
  block_sum_max(s, mx);
  if (threadIdx.x == 0) {
    if (mean) *mean = s;
    if (absmax) *absmax = __longlong_as_double((long long)mx);
  }
}

// ---------------------------------------------------------------------------
// Tangential derivatives (Section 4, Differentiation, eqs. diff_x..diff_z and
// Msin) on the folded coefficients X[j][k] of coeffs2 (the paper's convention:
// coefficients of e^{ij theta} e^{ik lambda}, j in [0, N), k in [0, L], with
// X_{-j,k} = (-1)^k X_{j,k}; the lambda-Nyquist column k = L is dropped).
//
// Q = (1/sin theta) d/dlambda f in coefficients: M_sin Q = a with a = ik X
// (eq. Msin: (i/2)(x_{j+1} - x_{j-1}) = a_j).  A quotient by sin theta of a
// function on the sphere has the symmetry Q_{-j,k} = -(-1)^k Q_{j,k} (the
// numerator is BMC, sin theta is odd in theta), so only j >= 0 is formed, and
// the rows of M_sin that the folded unknowns can satisfy fix it:
//   k odd  (Q_{-j} = Q_j):  rows j = 1..N-1 with x_N = x_{N-1} = 0, run down
//          from the top: x_{j-1} = x_{j+1} + 2i a_j, i.e.
//          x_j = 2i sum_{r = j+1, j+3, ... <= N-1} a_r = -2k sum_r X_{r,k};
//   k even (Q_{-j} = -Q_j, so x_0 = 0):  rows j = 0..N-2 run up from the
//          bottom, row 0 reading -2 x_1 = 2i a_0: x_{j+1} = x_{j-1} - 2i a_j, i.e.
//          x_j = -2i sum_{r = j-1, j-3, ... >= 0} w_r a_r = 2k sum_r w_r X_{r,k}
//          with w_0 = 1/2, w_r = 1 otherwise.
// This is the part with that symmetry of the dense solve of M_sin on the
// m-point window j in [-m/2, m/2-1] (for odd k the solve has the symmetry
// already; for even k the window's asymmetric bottom row leaves a part
// without it, which the samples on theta > 0 do not see), and M_sin^{-1} a
// itself whenever the quotient lies in the window (band-limited f).
// The sums are taken over row chunks of kMsinRows rows so that every
// (chunk, column) has a thread: pass 1 sums each chunk's even and odd rows into
// P[2c][k], P[2c+1][k] (row 0 weighted 1/2 in even columns); a scan turns those
// into the sums over the chunks above (odd k) or below (even k), one thread per
// column and parity; pass 3 walks each chunk, downwards for odd k and upwards for
// even k, writing Q and carrying the sums already scaled by -/+2k (one FMA per
// coefficient).
// Grid of passes 1 and 3: (ceil(Kp / blockDim.x), chunks).
// ---------------------------------------------------------------------------
constexpr int kMsinRows = 64;

__global__ void k_msin_partial(const cpx<double>* __restrict__ X, cpx<double>* __restrict__ P, int N, int K,
                               int Kp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Kp) return;
  const int c = blockIdx.y, j0 = c * kMsinRows, j1 = min(N, j0 + kMsinRows);
  cpx<double> se = {0.0, 0.0}, so = {0.0, 0.0};
  if (k < K - 1) {                           // k = L (Nyquist) and padding columns are zero
#pragma unroll 4
    for (int j = j0; j < j1; j += 2) {       // j0 is even
      se = se + X[(size_t)j * Kp + k];
      if (j + 1 < j1) so = so + X[(size_t)(j + 1) * Kp + k];
    }
    if (c == 0 && (k & 1) == 0) se = se - 0.5 * X[k];   // w_0 = 1/2 in even columns
  }
  P[(size_t)(2 * c) * Kp + k] = se;
  P[(size_t)(2 * c + 1) * Kp + k] = so;
}

// P[2c + par][k] <- the sum of the chunk sums over the chunks c' > c (odd k) or
// c' < c (even k): an exclusive scan in the direction that column's walk takes
__global__ void k_msin_scan(cpx<double>* __restrict__ P, int chunks, int Kp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * Kp) return;
  const int par = idx >= Kp, k = par ? idx - Kp : idx;
  const bool up = (k & 1) == 0;
  cpx<double> run = {0.0, 0.0};
  for (int t = 0; t < chunks; ++t) {
    const int c = up ? t : chunks - 1 - t;
    cpx<double>& slot = P[(size_t)(2 * c + par) * Kp + k];
    const cpx<double> v = slot;
    slot = run;
    run = run + v;
  }
}

__global__ void k_msin_apply(const cpx<double>* __restrict__ X, const cpx<double>* __restrict__ P,
                             cpx<double>* __restrict__ Q, int N, int K, int Kp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Kp) return;
  const int c = blockIdx.y, j0 = c * kMsinRows, j1 = min(N, j0 + kMsinRows);
  const bool live = k < K - 1;
  const bool up = (k & 1) == 0;
  const double scale = up ? 2.0 * (double)k : -2.0 * (double)k;
  // the scaled sums of the even / odd rows beyond this chunk in the walk's direction
  cpx<double> se = {0.0, 0.0}, so = {0.0, 0.0};
  if (live) {
    se = scale * P[(size_t)(2 * c) * Kp + k];
    so = scale * P[(size_t)(2 * c + 1) * Kp + k];
  }
  const int len = j1 - j0;
#pragma unroll 4
  for (int t = 0; t < len; ++t) {
    const int j = up ? j0 + t : j1 - 1 - t;
    // Q_j takes the rows of the other parity already walked past
    Q[(size_t)j * Kp + k] = (j & 1) ? se : so;
    if (live) {
      const cpx<double> x = X[(size_t)j * Kp + k];
      const double sc = (up && j == 0) ? 0.5 * scale : scale;
      cpx<double>& s = (j & 1) ? so : se;
      s = {fma(sc, x.re, s.re), fma(sc, x.im, s.im)};
    }
  }
}

// Coefficient chop (the derivative operators' optional truncation): the
// coefficients with |X_jk| <= rtol max |X| are set to zero before the maps act,
// so that rounding noise in modes a band-limited input does not have is not
// amplified by the division by sin theta.  Live columns k < K - 1 only; grid
// (ceil(Kp / blockDim.x), rows) with the rows striding over j.
// max |X_jk|^2 into *mx as the bits of a non-negative double (atomicMax on the
// bit pattern orders non-negative doubles); blockDim.x a multiple of 32
__global__ void k_coeff_absmax(const cpx<double>* __restrict__ X, int N, int K, int Kp,
                               unsigned long long* __restrict__ mx) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (k < K - 1) {
    for (int j = blockIdx.y; j < N; j += gridDim.y) {
      const cpx<double> v = X[(size_t)j * Kp + k];
      m = fmax(m, fma(v.re, v.re, v.im * v.im));
    }
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    atomicMax(mx, (unsigned long long)__double_as_longlong(t));
  }
}
// zero |X_jk|^2 <= rtol^2 max |X|^2
__global__ void k_coeff_chop(cpx<double>* __restrict__ X, int N, int K, int Kp,
                             const unsigned long long* __restrict__ mx, double rtol) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K - 1) return;
  const double thr = rtol * rtol * __longlong_as_double((long long)*mx);
  for (int j = blockIdx.y; j < N; j += gridDim.y) {
    cpx<double>& v = X[(size_t)j * Kp + k];
    const cpx<double> x = v;
    if (fma(x.re, x.re, x.im * x.im) <= thr) v = {0.0, 0.0};
  }
}

// x with its sign flipped when c is set: an integer operation on the sign bit,
// which keeps conditional negations off the FP64 pipe
__device__ __forceinline__ double flip_if(double x, bool c) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)c << 63));
}
// X_{i,k} for i in [-1, N] (the BMC mirror at i = -1, zero at i = N and in the
// Nyquist column)
__device__ __forceinline__ cpx<double> x_at(const cpx<double>* __restrict__ X, int i, int k, int N, int K,
                                            int Kp) {
  const bool mirror = i < 0;
  if (mirror) i = 1;
  if (k >= K - 1 || i >= N) return {0.0, 0.0};
  const cpx<double> v = X[(size_t)i * Kp + k];
  const bool f = mirror && (k & 1);
  return {flip_if(v.re, f), flip_if(v.im, f)};
}
// s C with C = cos theta d/dtheta f: C_j = (D_{j-1} + D_{j+1})/2, D_i = i i X_i;
// columns k = -1 by the real-function symmetry C_{j,-1} = conj(C_{j,1}).
// wm = s (j-1)/2, wp = s (j+1)/2.
__device__ __forceinline__ cpx<double> c_at(const cpx<double>* __restrict__ X, int j, int k, int N, int K,
                                            int Kp, double wm, double wp) {
  const int kk = k < 0 ? 1 : k;
  const cpx<double> a = x_at(X, j - 1, kk, N, K, Kp), b = x_at(X, j + 1, kk, N, K, Kp);
  // i (wm a + wp b), conjugated for k = -1
  const cpx<double> t = {fma(wm, a.re, wp * b.re), fma(wm, a.im, wp * b.im)};
  return {-t.im, flip_if(t.re, k < 0)};
}
__device__ __forceinline__ cpx<double> q_at(const cpx<double>* __restrict__ Q, int j, int k, int K, int Kp) {
  if (k >= K - 1) return {0.0, 0.0};
  const bool c = k < 0;
  const cpx<double> v = Q[(size_t)j * Kp + (c ? 1 : k)];
  return {v.re, flip_if(v.im, c)};
}

// Coefficients of the Cartesian components of the surface gradient:
//   T0: d^t/dx = -sin(lambda) Q + cos(lambda) C
//   T1: d^t/dy =  cos(lambda) Q + sin(lambda) C
//   T2: d^t/dz = -sin(theta) d/dtheta f, T2_j = ((j+1) X_{j+1} - (j-1) X_{j-1})/2
//       (the chain-rule sign for the colatitude theta)
// with cos(lambda) g -> (g_{k-1} + g_{k+1})/2, sin(lambda) g -> (i/2)(g_{k+1} - g_{k-1}).
// One launch forms up to three outputs from one input, output o receiving
// +-T_{comp[o]}, added to its contents when bit o of ACC is set: the gradient
// (three outputs), a divergence term or two curl terms; T0 and T1 share their
// loads and sums.  Thread per (j, k), grid (ceil(Kp / blockDim.x), rows) with
// the rows striding over j; the Nyquist and padding columns receive zero terms.
// ---------------------------------------------------------------------------
// (the launch descriptor TangentialCombo is declared with the batched-plan types)
template <int ACC>
__global__ void k_tangential(const cpx<double>* __restrict__ X, const cpx<double>* __restrict__ Q,
                             const TangentialCombo tc, int N, int K, int Kp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Kp) return;
  const bool live = k < K - 1;
  for (int j = blockIdx.y; j < N; j += gridDim.y) {
    cpx<double> T0 = {0.0, 0.0}, T1 = {0.0, 0.0}, T2 = {0.0, 0.0};
    if (live) {
      const double wm = fma(0.5, (double)j, -0.5), wp = wm + 1.0;   // (j -+ 1)/2
      if (tc.need_xy) {
        const cpx<double> qp = q_at(Q, j, k + 1, K, Kp), qm = q_at(Q, j, k - 1, K, Kp);
        // C/2 at k +- 1 (half weights), so that T0 and T1 take one FMA per part
        const double hm = 0.5 * wm, hp = 0.5 * wp;
        const cpx<double> cp = c_at(X, j, k + 1, N, K, Kp, hm, hp), cm = c_at(X, j, k - 1, N, K, Kp, hm, hp);
        const cpx<double> dq = qp - qm, sc = cp + cm, sq = qp + qm, dc = cp - cm;
        T0 = {fma(0.5, dq.im, sc.re), fma(-0.5, dq.re, sc.im)};   // -(i/2) dq + (cp + cm)/2
        T1 = {fma(0.5, sq.re, -dc.im), fma(0.5, sq.im, dc.re)};   // sq/2 + (i/2)(cp - cm)
      }
      if (tc.need_z) {
        const cpx<double> a = x_at(X, j + 1, k, N, K, Kp), b = x_at(X, j - 1, k, N, K, Kp);
        T2 = {fma(wp, a.re, -wm * b.re), fma(wp, a.im, -wm * b.im)};
      }
    }
    const size_t o = (size_t)j * Kp + k;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      if (!tc.G[g]) continue;
      const int c = tc.comp[g];
      cpx<double> t = c == 0 ? T0 : (c == 1 ? T1 : T2);
      const bool ng = tc.neg[g] != 0;
      t = {flip_if(t.re, ng), flip_if(t.im, ng)};
      if (ACC & (1 << g)) t = tc.G[g][o] + t;
      tc.G[g][o] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// Pointwise products with the unit normal n = (x, y, z) of eq.
// sphericalCoordinates, x = cos(lambda) sin(theta), y = sin(lambda) sin(theta),
// z = cos(theta), on the n_theta x n_lambda grid.  geo holds sin(theta_i),
// cos(theta_i) (n_theta each), then cos(lambda_q), sin(lambda_q) (n_lambda
// each).  Grid (ceil(n_lambda / blockDim.x), rows), rows striding over i.
// ---------------------------------------------------------------------------
struct Normal {
  double x, y, z;
};
__device__ __forceinline__ Normal normal_at(const double* __restrict__ geo, int nt, int nl, int i, int q) {
  const double st = geo[i], ct = geo[nt + i], cl = geo[2 * nt + q], sl = geo[2 * nt + nl + q];
  return {cl * st, sl * st, ct};
}
// (a, b, c) <- n x (a, b, c): the curl of a scalar function (eq. CurlScalarF)
// from its gradient
__global__ void k_cross_normal(double* __restrict__ a, double* __restrict__ b, double* __restrict__ c,
                               const double* __restrict__ geo, int nt, int nl) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nl) return;
  for (int i = blockIdx.y; i < nt; i += gridDim.y) {
    const Normal n = normal_at(geo, nt, nl, i, q);
    const size_t o = (size_t)i * nl + q;
    const double va = a[o], vb = b[o], vc = c[o];
    a[o] = n.y * vc - n.z * vb;
    b[o] = n.z * va - n.x * vc;
    c[o] = n.x * vb - n.y * va;
  }
}
// out = x a + y b + z c (the vorticity from the curl); out may be c
__global__ void k_normal_dot(const double* __restrict__ a, const double* __restrict__ b, const double* c,
                             double* out, const double* __restrict__ geo, int nt, int nl) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nl) return;
  for (int i = blockIdx.y; i < nt; i += gridDim.y) {
    // sin(theta) (cos(lambda) a + sin(lambda) b) + cos(theta) c
    const double st = geo[i], ct = geo[nt + i], cl = geo[2 * nt + q], sl = geo[2 * nt + nl + q];
    const size_t o = (size_t)i * nl + q;
    out[o] = fma(st, fma(cl, a[o], sl * b[o]), ct * c[o]);
  }
}

// ---------------------------------------------------------------------------
// Structure-preserving GE (Section 3, Figure GaussianElimination) on the
// residual e[i][q] of the theta > 0 half of the DFS grid (the residual stays
// BMC, so the other half is e(lambda, -theta) = e(lambda + pi, theta)).
// A term t is a column c_t(theta_p) = e(lambda* - pi, theta_p) on the full DFS
// grid (m = 2 n_theta samples), a row r_t(lambda_q) = e(lambda_q, theta*) and
// the entries (P00, P01) of the centrosymmetric epsilon-pseudoinverse of the
// pivot matrix; the term is [c(theta) c(-theta)] P [r(lambda); r(lambda + pi)].
// ---------------------------------------------------------------------------
// (the pivot record GePivot is declared with the batched-plan types)
// per-block partial maxima over the search region theta_i > 0 (all i),
// lambda_q in [0, pi) (q >= n/2) and max |e| over all entries
__global__ void k_ge_pivot_partial(const double* __restrict__ e, int nt, int n, GePivot* __restrict__ part) {
  const int H = n >> 1;
  const long long total = (long long)nt * H;
  double best = -1.0, mx = 0.0;
  long long bi = 0;
  // t = i H + qq, advanced by the grid stride without a division per element
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int di = (int)(stride / H), dq = (int)(stride - (long long)di * H);
  int i = (int)(t0 / H), qq = (int)(t0 - (long long)i * H);
  for (long long t = t0; t < total; t += stride) {
    const double a = e[(size_t)i * n + qq], b = e[(size_t)i * n + qq + H];
    // sigma_1 of [[a, b], [b, a]] = max |a +- b| = |a| + |b|
    const double s1 = fabs(a) + fabs(b);
    if (s1 > best) {
      best = s1;
      bi = t;
    }
    mx = fmax(mx, fmax(fabs(a), fabs(b)));
    i += di;
    qq += dq;
    if (qq >= H) {
      qq -= H;
      ++i;
    }
  }
  __shared__ double sb[32], sm[32];
  __shared__ long long si[32];
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const long long oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  }
  if ((threadIdx.x & 31) == 0) {
    sb[threadIdx.x >> 5] = best;
    si[threadIdx.x >> 5] = bi;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (sb[w] > best || (sb[w] == best && si[w] < bi)) {
        best = sb[w];
        bi = si[w];
      }
      mx = fmax(mx, sm[w]);
    }
    part[blockIdx.x] = GePivot{best, 0.0, 0.0, mx, bi};
  }
}

// one thread: reduce the partials, read the pivot's a and b
// one CTA (blockDim.x a multiple of 32): the best partial (smallest index among
// ties) and the maximum, then the pivot's two entries
__global__ void k_ge_pivot_final(const double* __restrict__ e, int n, const GePivot* __restrict__ part, int nparts,
                                 GePivot* __restrict__ out) {
  double best = -1.0, mx = 0.0;
  long long bi = 0x7fffffffffffffffLL;
  for (int w = threadIdx.x; w < nparts; w += blockDim.x) {
    const GePivot o = part[w];
    if (o.best > best || (o.best == best && o.index < bi)) {
      best = o.best;
      bi = o.index;
    }
    mx = fmax(mx, o.maxabs);
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const long long oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  }
  __shared__ double sb[32], sm[32];
  __shared__ long long si[32];
  if ((threadIdx.x & 31) == 0) {
    sb[threadIdx.x >> 5] = best;
    si[threadIdx.x >> 5] = bi;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (sb[w] > best || (sb[w] == best && si[w] < bi)) {
        best = sb[w];
        bi = si[w];
      }
      mx = fmax(mx, sm[w]);
    }
    const int H = n >> 1;
    const int i = (int)(bi / H), qq = (int)(bi - (long long)i * H);
    *out = GePivot{best, e[(size_t)i * n + qq], e[(size_t)i * n + qq + H], mx, bi};
  }
}

// copy the term's column (full DFS grid, m = 2 nt) and row out of the residual:
// c(theta_p) = e(lambda* - pi, theta_p): for p >= nt, e[p - nt][q* - n/2]; for
// p < nt (theta_p = -theta_{nt-1-p}), e(lambda*, theta_{nt-1-p}) = e[nt-1-p][q*]
// the step's column and row of e, and the row's two pivot combinations
// A_q = p0 r(lambda_q) + p1 r(lambda_q + pi), B_q = p1 r(lambda_q) + p0 r(lambda_q + pi)
__global__ void k_ge_extract(const double* __restrict__ e, int nt, int n, int istar, int qstar,
                             double* __restrict__ col, double* __restrict__ row, double p0, double p1,
                             double* __restrict__ AB) {
  const int H = n >> 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 2 * nt) {
    const int p = t;
    col[p] = p >= nt ? e[(size_t)(p - nt) * n + (qstar - H)] : e[(size_t)(nt - 1 - p) * n + qstar];
  }
  if (t < n) {
    const double r0 = e[(size_t)istar * n + t], r1 = e[(size_t)istar * n + (t < H ? t + H : t - H)];
    row[t] = r0;
    AB[t] = fma(p0, r0, p1 * r1);
    AB[n + t] = fma(p1, r0, p0 * r1);
  }
}

// e[i][q] -= c(theta_i) A_q + c(-theta_i) B_q; grid (ceil(n / blockDim.x), rows),
// the rows striding over i so that each thread keeps its A_q, B_q
__global__ void k_ge_update(double* __restrict__ e, int nt, int n, const double* __restrict__ col,
                            const double* __restrict__ AB) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double A = AB[q], B = AB[n + q];
  for (int i = blockIdx.y; i < nt; i += gridDim.y) {
    const double cp = col[nt + i], cm = col[nt - 1 - i];
    double& v = e[(size_t)i * n + q];
    v = fma(-cp, A, fma(-cm, B, v));
  }
}

// ---------------------------------------------------------------------------
// Low-rank right-hand side: F = coefficients of sin^2(theta) f~ from the terms.
// With the column's symmetric and antisymmetric parts s_t, a_t (coefficients
// S_t, A_t from theta_forward) and the row's longitude coefficients R_t, the
// term [c(theta) c(-theta)] P [r(lambda); r(lambda + pi)] has coefficients
//   F_jk = 2 (P00 + P01) S_t,j R_t,k (k even),  2 (P00 - P01) A_t,j R_t,k (k odd)
// since c(-theta) has coefficients S - A and r(lambda + pi) has (-1)^k R.
// ---------------------------------------------------------------------------
// packed columns for theta_forward: Wc[i][2t] = sin^2(theta_i) (c(theta_i) + c(-theta_i))/2,
// Wc[i][2t+1] = sin^2(theta_i) (c(theta_i) - c(-theta_i))/2  (Kc = 2 * terms columns)
__global__ void k_lowrank_pack(const double* __restrict__ cols, int terms, int nt, const double* __restrict__ sin2,
                               cpx<double>* __restrict__ Wc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nt * terms) return;
  const int i = idx / terms, t = idx - i * terms;
  const double* c = cols + (size_t)t * 2 * nt;
  const double cp = c[nt + i], cm = c[nt - 1 - i], w = 0.5 * sin2[i];
  Wc[(size_t)i * 2 * terms + 2 * t] = {w * (cp + cm), 0.0};
  Wc[(size_t)i * 2 * terms + 2 * t + 1] = {w * (cp - cm), 0.0};
}

// fold the pivot weights into the packed coefficients, in place:
// Wc[j][2t] = 2(P00 + P01) S_t,j, Wc[j][2t+1] = 2(P00 - P01) A_t,j
__global__ void k_lowrank_weights(cpx<double>* __restrict__ Wc, const double* __restrict__ piv, int terms, int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * terms) return;
  const int j = idx / terms, t = idx - j * terms;
  const double p0 = piv[2 * t], p1 = piv[2 * t + 1];
  const double we = 2.0 * (p0 + p1), wo = 2.0 * (p0 - p1);
  cpx<double>* z = Wc + (size_t)j * 2 * terms + 2 * t;
  z[0] = we * z[0];
  z[1] = wo * z[1];
}

// F[j][k] = sum_t Wc[j][2t + (k & 1)] R[t][k]: one CTA per row j (its 2 * terms
// weighted coefficients in shared memory), one thread per k; k >= K written as zero
__global__ void k_lowrank_outer(const cpx<double>* __restrict__ Wc, const cpx<double>* __restrict__ R, int terms,
                                int K, int Kp, cpx<double>* __restrict__ F) {
  extern __shared__ cpx<double> zrow[];
  const int j = blockIdx.y;
  for (int s = threadIdx.x; s < 2 * terms; s += blockDim.x) zrow[s] = Wc[(size_t)j * 2 * terms + s];
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Kp) return;
  cpx<double> acc = {0.0, 0.0};
  if (k < K) {
    const cpx<double>* z = zrow + (k & 1);
#pragma unroll 4
    for (int t = 0; t < terms; ++t) {
      const cpx<double> zt = z[2 * t], rt = R[(size_t)t * Kp + k];
      acc = {fma(zt.re, rt.re, fma(-zt.im, rt.im, acc.re)), fma(zt.re, rt.im, fma(zt.im, rt.re, acc.im))};
    }
  }
  F[(size_t)j * Kp + k] = acc;
}

}  // namespace sp
