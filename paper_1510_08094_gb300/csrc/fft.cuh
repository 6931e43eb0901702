// Shared-memory mixed-radix FFT used by every transform stage.
//
// One CTA transforms `nbatch` sequences of length L = R_1 R_2 ... R_s that sit
// back to back in shared memory, in place, by decimation in time: the input is
// loaded in mixed-radix digit-reversed order, pass t combines R_t sub-DFTs of
// length Ns = R_1 ... R_{t-1}, and the output comes out in natural order.
// Twiddles come from a per-pass table laid out so that one butterfly's R
// twiddles are adjacent (one or a few vector loads, coalesced across the
// threads of a pass); the odd-prime DFT constants follow the pass tables.
#pragma once

#include <cuda_runtime.h>

#include "dd.cuh"
#include <type_traits>

namespace sp {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
  T re, im;
};

template <typename T> __device__ __forceinline__ cpx<T> mk(T a, T b) { return cpx<T>{a, b}; }
template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return {a.re, -a.im}; }
// x, negated when c is set, by flipping the sign bit(s) with integer operations:
// a runtime-conditional negation written as a select between x and -x costs an
// FP64 (or FP32) add per element, on GB300's narrow FP64 pipe a real cost
__device__ __forceinline__ double neg_if(double x, bool c) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)c << 63));
}
__device__ __forceinline__ float neg_if(float x, bool c) {
  return __int_as_float(__float_as_int(x) ^ ((int)c << 31));
}
__device__ __forceinline__ dd neg_if(dd x, bool c) { return dd(neg_if(x.hi, c), neg_if(x.lo, c)); }
template <typename T> __device__ __forceinline__ cpx<T> neg_if(cpx<T> a, bool c) {
  return {neg_if(a.re, c), neg_if(a.im, c)};
}
// a * b
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return {fma(a.re, b.re, a.im * b.im), fma(a.im, b.re, -a.re * b.im)};
}
// a * (-i) for DIR = -1, a * (+i) for DIR = +1
template <int DIR, typename T> __device__ __forceinline__ cpx<T> rot(cpx<T> a) {
  return DIR < 0 ? cpx<T>{a.im, -a.re} : cpx<T>{-a.im, a.re};
}
// a * w^DIR-sense: w from the forward table; inverse uses conj(w)
template <int DIR, typename T> __device__ __forceinline__ cpx<T> twmul(cpx<T> a, cpx<T> w) {
  return DIR < 0 ? cmul(a, w) : cmulc(a, w);
}

// read-only cached load of a table entry
__device__ __forceinline__ cpx<double> ldg_c(const cpx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cpx<float> ldg_c(const cpx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cpx<dd> ldg_c(const cpx<dd>* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {dd(v.x, v.y), dd(v.z, v.w)};
}

// conversions between the arithmetic type of a transform and double
template <typename T> struct num;
template <> struct num<double> {
  static __device__ __forceinline__ double from_double(double x) { return x; }
  static __device__ __forceinline__ double to_double(double x) { return x; }
};
template <> struct num<float> {
  static __device__ __forceinline__ float from_double(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ double to_double(float x) { return (double)x; }
};
template <> struct num<dd> {
  static __device__ __forceinline__ dd from_double(double x) { return dd_from_double(x); }
  static __device__ __forceinline__ double to_double(dd x) { return dd_to_double(x); }
};

constexpr int kMaxStages = 16;

// Unsigned division by an invariant divisor d (Granlund & Montgomery 1994,
// "Division by invariant integers using multiplication", Fig. 4.1):
// l = ceil(log2 d), m = floor(2^32 (2^l - d)/d) + 1, and then
// n / d = (t + ((n - t) >> min(l,1))) >> max(l-1,0) with t = umulhi(m, n).
struct FastDiv {
  unsigned m, s1, s2;
};
__host__ inline FastDiv make_fastdiv(unsigned d) {
  unsigned l = 0;
  while ((1ull << l) < d) ++l;
  unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return {(unsigned)m, l < 1 ? l : 1u, l > 1 ? l - 1 : 0u};
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  unsigned t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct FftDesc {
  int L;
  int nstages;
  int radix[kMaxStages];
  FastDiv div_L;               // n / L
  FastDiv div_nb[kMaxStages];  // n / (L / R_s)
  FastDiv div_ns[kMaxStages];  // n / (R_1 ... R_{s-1})
  // twiddle table: pass s (sub-DFT length Ns = R_1 ... R_{s-1}) holds at
  // tw_off[s] + k RP + r the value exp(-2 pi i r k / (Ns R_s)), r < R_s, k < Ns,
  // RP = R_s rounded up to even; for odd R_s >= 7, dft_off[s] + a holds
  // exp(-2 pi i a / R_s), a < R_s.  tw_len entries in all.
  int tw_off[kMaxStages];
  int dft_off[kMaxStages];
  // radix-2, 3, 4, 5 and 8 passes with Ns > 1: g_off[s] + 8 k holds butterfly
  // k's scaled twiddle record for the FP64 kernels (see fft_pass), else -1
  int g_off[kMaxStages];
  int tw_len;
};

// Scaled twiddle record of one radix-5 butterfly (16 doubles as 8 complex
// entries).  Each twiddle is written w_r = sigma_r (1 + i tau_r), or, where
// |Im w_r| > |Re w_r|, w_r = i sigma_r (1 + i tau_r), so |tau_r| <= 1 and
// |sigma_r| >= 1/sqrt2; the butterfly then forms x_r (1 + i tau_r) (two FMAs),
// rotates by i where flagged (sign-bit and register moves only), and carries the
// real scales sigma_r through the 5-point DFT as the ratios and products below,
// taken into its FMAs.
struct Radix5Record {
  double tau[4];        // tau_1 .. tau_4
  double q4, q3, rho;   // sigma_4/sigma_1, sigma_3/sigma_2, sigma_2/sigma_1
  double s1;            // sigma_1
  double s1q;           // sigma_1 / 4
  double q5s1;          // (sqrt5/4) sigma_1
  double rrho, rirho;   // r rho, rho / r  (r = sin(4 pi/5) / sin(2 pi/5))
  double ss1, ss2;      // sin(2 pi/5) sigma_1, sin(4 pi/5) sigma_1
  long long rot;        // bit r-1: w_r carries the factor i
  long long pad;
};
// The same for a radix-8 butterfly: the even inputs 0, 2, 4, 6 and the odd
// inputs 1, 3, 5, 7 form their 4-point DFTs with the scales as ratios, the odd
// half ending on the common scale sigma_1.
struct Radix8Record {
  double tau[7];        // tau_1 .. tau_7
  double s4;            // sigma_4
  double q62, s2;       // sigma_6/sigma_2, sigma_2
  double q51, q73, q31; // sigma_5/sigma_1, sigma_7/sigma_3, sigma_3/sigma_1
  double s1, s1h;       // sigma_1, sigma_1/sqrt2
  long long rot;        // bit r-1: w_r carries the factor i
};
// radix 4: x0 +- sigma_2 h2 and sigma_1 (h1 +- q31 h3)
struct Radix4Record {
  double tau[3];
  double s2, q31, s1;
  long long rot;
  double pad[9];
};
// radix 3: sigma_1 (h1 +- q21 h2), then the constants -1/2 and sin(2 pi/3) times sigma_1
struct Radix3Record {
  double tau[2];
  double q21, s1, s1half, ss1;
  long long rot;
  double pad[9];
};
// radix 2: x0 +- sigma_1 h1
struct Radix2Record {
  double tau, s1;
  long long rot;
  double pad[13];
};

// the twiddles w[r], 0 < r < R, of one butterfly from its R-entry slot p
template <int R, typename T>
__device__ __forceinline__ void load_stage_tw(const cpx<T>* __restrict__ p, cpx<T>* w) {
#pragma unroll
  for (int r = 1; r < R; ++r) w[r] = ldg_c(p + r);
}
// FP32: the slot is RP = even entries of 8 bytes starting on a 16-byte boundary,
// read as RP/2 16-byte loads
template <int R>
__device__ __forceinline__ void load_stage_tw(const cpx<float>* __restrict__ p, cpx<float>* w) {
  // w^1 and w^2 from the table (one 16-byte load), higher powers by products of
  // depth <= 2 (w^3 = w^2 w, w^4 = w^2 w^2, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3)
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  w[1] = {q.z, q.w};
  if constexpr (R > 2) {
    const float4 q2 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    w[2] = {q2.x, q2.y};
  }
  auto mul = [](cpx<float> a, cpx<float> b) {
    return cpx<float>{fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re)};
  };
  if constexpr (R > 3) w[3] = mul(w[2], w[1]);
  if constexpr (R > 4) w[4] = mul(w[2], w[2]);
  if constexpr (R > 5) w[5] = mul(w[4], w[1]);
  if constexpr (R > 6) w[6] = mul(w[4], w[2]);
  if constexpr (R > 7) w[7] = mul(w[4], w[3]);
}

// ---------------------------------------------------------------------------
// R-point DFTs on registers: y_a = sum_b x_b exp(DIR 2 pi i a b / R)
// ---------------------------------------------------------------------------

template <int DIR, typename T>
__device__ __forceinline__ void dft2(cpx<T>* v) {
  cpx<T> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <int DIR, typename T>
__device__ __forceinline__ void dft4(cpx<T>* v) {
  cpx<T> s0 = v[0] + v[2], d0 = v[0] - v[2];
  cpx<T> s1 = v[1] + v[3], d1 = rot<DIR>(v[1] - v[3]);
  v[0] = s0 + s1;
  v[2] = s0 - s1;
  v[1] = d0 + d1;
  v[3] = d0 - d1;
}

// In the butterflies below a constant factor of a term that is only added to
// or subtracted from another is folded into the final additions as FMAs
// (y = t +- i s w with s real: y.re = fma(-+s, w.im, t.re), ...), which saves
// the separate multiplications on the FP64 pipe.
template <int DIR, typename T>
__device__ __forceinline__ void dft8(cpx<T>* v) {
  const T h = (T)0.70710678118654752440084436210484903928;
  cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
  // 4-point DFTs of the even and odd samples (inputs in natural order 0,1,2,3)
  {
    cpx<T> s0 = e[0] + e[2], d0 = e[0] - e[2], s1 = e[1] + e[3], d1 = rot<DIR>(e[1] - e[3]);
    e[0] = s0 + s1; e[2] = s0 - s1; e[1] = d0 + d1; e[3] = d0 - d1;
  }
  {
    cpx<T> s0 = o[0] + o[2], d0 = o[0] - o[2], s1 = o[1] + o[3], d1 = rot<DIR>(o[1] - o[3]);
    o[0] = s0 + s1; o[2] = s0 - s1; o[1] = d0 + d1; o[3] = d0 - d1;
  }
  // twiddles W8^k (DIR sense): W8^1 = (1 + DIR i)/sqrt2, W8^2 = DIR i, W8^3 = (-1 + DIR i)/sqrt2:
  //   W8^1 o1 = h (p1, q1),  W8^3 o3 = h (ha p3, hb q3) with the signs ha, hb
  //   (DIR < 0: ( o3.im - o3.re, -(o3.re + o3.im)); DIR > 0: (-(o3.re + o3.im), o3.re - o3.im))
  const T p1 = DIR < 0 ? o[1].re + o[1].im : o[1].re - o[1].im;
  const T q1 = DIR < 0 ? o[1].im - o[1].re : o[1].im + o[1].re;
  const T p3 = DIR < 0 ? o[3].im - o[3].re : o[3].re + o[3].im;
  const T q3 = DIR < 0 ? o[3].re + o[3].im : o[3].re - o[3].im;
  const T ha = DIR < 0 ? h : -h, hb = DIR < 0 ? -h : h;
  cpx<T> t2 = rot<DIR>(o[2]);
  v[0] = e[0] + o[0]; v[4] = e[0] - o[0];
  v[1] = {fma(h, p1, e[1].re), fma(h, q1, e[1].im)};
  v[5] = {fma(-h, p1, e[1].re), fma(-h, q1, e[1].im)};
  v[2] = e[2] + t2;   v[6] = e[2] - t2;
  v[3] = {fma(ha, p3, e[3].re), fma(hb, q3, e[3].im)};
  v[7] = {fma(-ha, p3, e[3].re), fma(-hb, q3, e[3].im)};
}

// y = t + DIR i s w and y' = t - DIR i s w for real s
template <int DIR, typename T>
__device__ __forceinline__ void plus_minus_i(cpx<T> t, T s, cpx<T> w, cpx<T>& y, cpx<T>& yc) {
  const T g = DIR < 0 ? s : -s;              // DIR i s w = (-DIR s w.im, DIR s w.re)
  y = {fma(g, w.im, t.re), fma(-g, w.re, t.im)};
  yc = {fma(-g, w.im, t.re), fma(g, w.re, t.im)};
}

template <int DIR, typename T>
__device__ __forceinline__ void dft3(cpx<T>* v) {
  const T c = (T)-0.5;
  const T s = (T)0.86602540378443864676372317075293618347;  // sin(2 pi / 3)
  cpx<T> a = v[1] + v[2], b = v[1] - v[2];
  cpx<T> t = {fma(c, a.re, v[0].re), fma(c, a.im, v[0].im)};
  v[0] = v[0] + a;
  // y1 = t + DIR i s b, y2 = t - DIR i s b
  plus_minus_i<DIR>(t, s, b, v[1], v[2]);
}

// 5 points with cos(2 pi/5) = (sqrt5 - 1)/4, cos(4 pi/5) = -(sqrt5 + 1)/4:
//   y0 = x0 + S, t1,2 = x0 - S/4 +- (sqrt5/4) D  (S = a1 + a2, D = a1 - a2),
//   y1,4 = t1 +- DIR i s1 (b1 + r b2), y2,3 = t2 +- DIR i s2 (b1 - b2 / r),
// s1 = sin(2 pi/5), s2 = sin(4 pi/5), r = s2/s1 = (sqrt5 - 1)/2.
template <int DIR, typename T>
__device__ __forceinline__ void dft5(cpx<T>* v) {
  const T q5 = (T)0.55901699437494742410229341718281905886;   // sqrt5 / 4
  const T s1 = (T)0.95105651629515357211643933337938214340;   // sin(2 pi/5)
  const T s2 = (T)0.58778525229247312916870595463907276860;   // sin(4 pi/5)
  const T r = (T)0.61803398874989484820458683436563811772;    // s2 / s1
  const T ri = (T)1.61803398874989484820458683436563811772;   // s1 / s2
  cpx<T> a1 = v[1] + v[4], b1 = v[1] - v[4];
  cpx<T> a2 = v[2] + v[3], b2 = v[2] - v[3];
  cpx<T> x0 = v[0];
  cpx<T> S = a1 + a2, D = a1 - a2;
  cpx<T> m = {fma((T)-0.25, S.re, x0.re), fma((T)-0.25, S.im, x0.im)};
  cpx<T> t1 = {fma(q5, D.re, m.re), fma(q5, D.im, m.im)};
  cpx<T> t2 = {fma(-q5, D.re, m.re), fma(-q5, D.im, m.im)};
  cpx<T> w1 = {fma(r, b2.re, b1.re), fma(r, b2.im, b1.im)};
  cpx<T> w2 = {fma(-ri, b2.re, b1.re), fma(-ri, b2.im, b1.im)};
  v[0] = x0 + S;
  plus_minus_i<DIR>(t1, s1, w1, v[1], v[4]);
  plus_minus_i<DIR>(t2, s2, w2, v[2], v[3]);
}

// Generic odd R: pair outputs a and R-a, using p_b = x_b + x_{R-b}, q_b = x_b - x_{R-b}.
// Cos/sin of 2 pi a b / R are read from the R-entry constant table dtw at a b mod R.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_odd(cpx<T>* v, const cpx<T>* __restrict__ dtw) {
  constexpr int H = (R - 1) / 2;
  cpx<T> p[H], q[H];
#pragma unroll
  for (int b = 1; b <= H; ++b) {
    p[b - 1] = v[b] + v[R - b];
    q[b - 1] = v[b] - v[R - b];
  }
  cpx<T> x0 = v[0];
  cpx<T> y0 = x0;
#pragma unroll
  for (int b = 0; b < H; ++b) y0 = y0 + p[b];
#pragma unroll
  for (int a = 1; a <= H; ++a) {
    cpx<T> A = x0, B = {(T)0, (T)0};
#pragma unroll
    for (int b = 1; b <= H; ++b) {
      cpx<T> w = ldg_c(dtw + (a * b) % R);
      T c = w.re, s = -w.im;  // w = exp(-2 pi i ab/R) = c - i s
      A.re = fma(c, p[b - 1].re, A.re);
      A.im = fma(c, p[b - 1].im, A.im);
      B.re = fma(s, q[b - 1].re, B.re);
      B.im = fma(s, q[b - 1].im, B.im);
    }
    // y_a = A + DIR i B, y_{R-a} = A - DIR i B
    cpx<T> iB = DIR < 0 ? cpx<T>{B.im, -B.re} : cpx<T>{-B.im, B.re};
    v[a] = A + iB;
    v[R - a] = A - iB;
  }
  v[0] = y0;
}

// ---------------------------------------------------------------------------
// Double-float butterflies: the same formulas, with every value that only
// feeds further operations of the butterfly kept unnormalised (dd.cuh) and
// every output normalised before it is stored.  The twiddle products are left
// unnormalised too: they feed the DFT (decimation in time), or are normalised
// by the decimation-in-frequency pass that stores them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ cpx<dd> cdd_add(cpx<dd> a, cpx<dd> b) { return {dd_add_u(a.re, b.re), dd_add_u(a.im, b.im)}; }
__device__ __forceinline__ cpx<dd> cdd_sub(cpx<dd> a, cpx<dd> b) { return {dd_sub_u(a.re, b.re), dd_sub_u(a.im, b.im)}; }
__device__ __forceinline__ cpx<dd> cdd_norm(cpx<dd> a) { return {dd_norm(a.re), dd_norm(a.im)}; }
// s x + t for a real double-float s
__device__ __forceinline__ cpx<dd> cdd_fmas(dd s, cpx<dd> x, cpx<dd> t) {
  return {dd_fma_u(s, x.re, t.re), dd_fma_u(s, x.im, t.im)};
}
__device__ __forceinline__ dd dd_flip(dd a) { return {-a.hi, -a.lo}; }
template <typename T> __device__ __forceinline__ cpx<T> out_norm(cpx<T> a) { return a; }
template <> __device__ __forceinline__ cpx<dd> out_norm<dd>(cpx<dd> a) { return cdd_norm(a); }

template <int DIR> __device__ __forceinline__ cpx<dd> twmul(cpx<dd> a, cpx<dd> w) {
  if (DIR < 0)   // a w
    return {dd_fma_u(a.re, w.re, dd_flip(dd_mul_u(a.im, w.im))), dd_fma_u(a.re, w.im, dd_mul_u(a.im, w.re))};
  // a conj(w)
  return {dd_fma_u(a.re, w.re, dd_mul_u(a.im, w.im)), dd_fma_u(a.im, w.re, dd_flip(dd_mul_u(a.re, w.im)))};
}

template <int DIR> __device__ __forceinline__ void dft2(cpx<dd>* v) {
  const cpx<dd> a = v[0], b = v[1];
  v[0] = cdd_norm(cdd_add(a, b));
  v[1] = cdd_norm(cdd_sub(a, b));
}

template <int DIR> __device__ __forceinline__ void dft4(cpx<dd>* v) {
  const cpx<dd> s0 = cdd_add(v[0], v[2]), d0 = cdd_sub(v[0], v[2]);
  const cpx<dd> s1 = cdd_add(v[1], v[3]), d1 = rot<DIR>(cdd_sub(v[1], v[3]));
  v[0] = cdd_norm(cdd_add(s0, s1));
  v[2] = cdd_norm(cdd_sub(s0, s1));
  v[1] = cdd_norm(cdd_add(d0, d1));
  v[3] = cdd_norm(cdd_sub(d0, d1));
}

// y = t + DIR i s w and y' = t - DIR i s w for real s, normalised
template <int DIR>
__device__ __forceinline__ void plus_minus_i(cpx<dd> t, dd s, cpx<dd> w, cpx<dd>& y, cpx<dd>& yc) {
  const dd g = DIR < 0 ? s : dd_flip(s);
  y = {dd_norm(dd_fma_u(g, w.im, t.re)), dd_norm(dd_fma_u(dd_flip(g), w.re, t.im))};
  yc = {dd_norm(dd_fma_u(dd_flip(g), w.im, t.re)), dd_norm(dd_fma_u(g, w.re, t.im))};
}

template <int DIR> __device__ __forceinline__ void dft3(cpx<dd>* v) {
  const dd c(-0.5), s(0.86602540378443864676372317075293618347);
  const cpx<dd> a = cdd_add(v[1], v[2]), b = cdd_sub(v[1], v[2]);
  const cpx<dd> t = cdd_fmas(c, a, v[0]);
  const cpx<dd> x0 = v[0];
  v[0] = cdd_norm(cdd_add(x0, a));
  plus_minus_i<DIR>(t, s, b, v[1], v[2]);
}

template <int DIR> __device__ __forceinline__ void dft5(cpx<dd>* v) {
  const dd q5(0.55901699437494742410229341718281905886), s1(0.95105651629515357211643933337938214340),
      s2(0.58778525229247312916870595463907276860), r(0.61803398874989484820458683436563811772),
      ri(1.61803398874989484820458683436563811772), quarter(-0.25);
  const cpx<dd> a1 = cdd_add(v[1], v[4]), b1 = cdd_sub(v[1], v[4]);
  const cpx<dd> a2 = cdd_add(v[2], v[3]), b2 = cdd_sub(v[2], v[3]);
  const cpx<dd> x0 = v[0];
  const cpx<dd> S = cdd_add(a1, a2), D = cdd_sub(a1, a2);
  const cpx<dd> m = cdd_fmas(quarter, S, x0);
  const cpx<dd> t1 = cdd_fmas(q5, D, m), t2 = cdd_fmas(dd_flip(q5), D, m);
  const cpx<dd> w1 = cdd_fmas(r, b2, b1), w2 = cdd_fmas(dd_flip(ri), b2, b1);
  v[0] = cdd_norm(cdd_add(x0, S));
  plus_minus_i<DIR>(t1, s1, w1, v[1], v[4]);
  plus_minus_i<DIR>(t2, s2, w2, v[2], v[3]);
}

template <int DIR> __device__ __forceinline__ void dft8(cpx<dd>* v) {
  const dd h(0.70710678118654752440084436210484903928);
  cpx<dd> e[4] = {v[0], v[2], v[4], v[6]};
  cpx<dd> o[4] = {v[1], v[3], v[5], v[7]};
  {
    const cpx<dd> s0 = cdd_add(e[0], e[2]), d0 = cdd_sub(e[0], e[2]), s1 = cdd_add(e[1], e[3]),
                  d1 = rot<DIR>(cdd_sub(e[1], e[3]));
    e[0] = cdd_add(s0, s1); e[2] = cdd_sub(s0, s1); e[1] = cdd_add(d0, d1); e[3] = cdd_sub(d0, d1);
  }
  {
    const cpx<dd> s0 = cdd_add(o[0], o[2]), d0 = cdd_sub(o[0], o[2]), s1 = cdd_add(o[1], o[3]),
                  d1 = rot<DIR>(cdd_sub(o[1], o[3]));
    o[0] = cdd_add(s0, s1); o[2] = cdd_sub(s0, s1); o[1] = cdd_add(d0, d1); o[3] = cdd_sub(d0, d1);
  }
  // as in the generic dft8: W8 o1 = h (p1, q1), W8^3 o3 = h (ha p3, hb q3)
  const dd p1 = DIR < 0 ? dd_add_u(o[1].re, o[1].im) : dd_sub_u(o[1].re, o[1].im);
  const dd q1 = DIR < 0 ? dd_sub_u(o[1].im, o[1].re) : dd_add_u(o[1].im, o[1].re);
  const dd p3 = DIR < 0 ? dd_sub_u(o[3].im, o[3].re) : dd_add_u(o[3].re, o[3].im);
  const dd q3 = DIR < 0 ? dd_add_u(o[3].re, o[3].im) : dd_sub_u(o[3].re, o[3].im);
  const dd ha = DIR < 0 ? h : dd_flip(h), hb = DIR < 0 ? dd_flip(h) : h;
  const cpx<dd> t2 = rot<DIR>(o[2]);
  v[0] = cdd_norm(cdd_add(e[0], o[0])); v[4] = cdd_norm(cdd_sub(e[0], o[0]));
  v[1] = {dd_norm(dd_fma_u(h, p1, e[1].re)), dd_norm(dd_fma_u(h, q1, e[1].im))};
  v[5] = {dd_norm(dd_fma_u(dd_flip(h), p1, e[1].re)), dd_norm(dd_fma_u(dd_flip(h), q1, e[1].im))};
  v[2] = cdd_norm(cdd_add(e[2], t2)); v[6] = cdd_norm(cdd_sub(e[2], t2));
  v[3] = {dd_norm(dd_fma_u(ha, p3, e[3].re)), dd_norm(dd_fma_u(hb, q3, e[3].im))};
  v[7] = {dd_norm(dd_fma_u(dd_flip(ha), p3, e[3].re)), dd_norm(dd_fma_u(dd_flip(hb), q3, e[3].im))};
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_any(cpx<T>* v, const cpx<T>* __restrict__ dtw) {
  if constexpr (R == 2) dft2<DIR>(v);
  else if constexpr (R == 3) dft3<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v);
  else if constexpr (R == 5) dft5<DIR>(v);
  else if constexpr (R == 8) dft8<DIR>(v);
  else dft_odd<R, DIR>(v, dtw);  // 7
}

// ---------------------------------------------------------------------------
// One in-place decimation-in-time pass over all batches; ends with a barrier.
// Butterfly (g, k), k < Ns, owns the R elements g Ns R + k + r Ns, multiplies
// element r by w^(r k), w = exp(-+2 pi i/(Ns R)), and applies the R-point DFT.
// Butterflies of a pass touch disjoint elements, so threads stream through
// them holding only R values.
// ---------------------------------------------------------------------------
// the radix-5 butterfly on the scaled record (FP64; see Radix5Record): the same
// outputs as twiddle multiplication followed by dft5, with 40 FP64 operations
// instead of 48
template <int DIR>
__device__ __forceinline__ void radix5_scaled(cpx<double>* v, const Radix5Record* __restrict__ rec) {
  const double2* q = reinterpret_cast<const double2*>(rec);
  const double2 t01 = __ldg(q), t23 = __ldg(q + 1), qq = __ldg(q + 2), rs = __ldg(q + 3);
  const double2 sq = __ldg(q + 4), rr = __ldg(q + 5), ss = __ldg(q + 6);
  const long long rot = __ldg(&rec->rot);
  const double tau[4] = {t01.x, t01.y, t23.x, t23.y};
  cpx<double> h[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    // the inverse transform uses conj(w): tau -> -tau and the factor i -> -i
    const double t = DIR < 0 ? tau[r] : -tau[r];
    const cpx<double> x = v[r + 1];
    const cpx<double> xt = {fma(-t, x.im, x.re), fma(t, x.re, x.im)};
    const bool rt = (rot >> r) & 1;
    // times i (forward) or -i (inverse) where flagged
    h[r] = {rt ? neg_if(xt.im, DIR < 0) : xt.re, rt ? neg_if(xt.re, DIR > 0) : xt.im};
  }
  const double q4 = qq.x, q3 = qq.y, rho = rs.x, s1 = rs.y, s1q = sq.x, q5s1 = sq.y;
  const double rrho = rr.x, rirho = rr.y, ss1 = ss.x, ss2 = ss.y;
  const cpx<double> a1 = {fma(q4, h[3].re, h[0].re), fma(q4, h[3].im, h[0].im)};
  const cpx<double> b1 = {fma(-q4, h[3].re, h[0].re), fma(-q4, h[3].im, h[0].im)};
  const cpx<double> a2 = {fma(q3, h[2].re, h[1].re), fma(q3, h[2].im, h[1].im)};
  const cpx<double> b2 = {fma(-q3, h[2].re, h[1].re), fma(-q3, h[2].im, h[1].im)};
  const cpx<double> S = {fma(rho, a2.re, a1.re), fma(rho, a2.im, a1.im)};
  const cpx<double> D = {fma(-rho, a2.re, a1.re), fma(-rho, a2.im, a1.im)};
  const cpx<double> x0 = v[0];
  v[0] = {fma(s1, S.re, x0.re), fma(s1, S.im, x0.im)};
  const cpx<double> m = {fma(-s1q, S.re, x0.re), fma(-s1q, S.im, x0.im)};
  const cpx<double> t1 = {fma(q5s1, D.re, m.re), fma(q5s1, D.im, m.im)};
  const cpx<double> t2 = {fma(-q5s1, D.re, m.re), fma(-q5s1, D.im, m.im)};
  const cpx<double> w1 = {fma(rrho, b2.re, b1.re), fma(rrho, b2.im, b1.im)};
  const cpx<double> w2 = {fma(-rirho, b2.re, b1.re), fma(-rirho, b2.im, b1.im)};
  plus_minus_i<DIR>(t1, ss1, w1, v[1], v[4]);
  plus_minus_i<DIR>(t2, ss2, w2, v[2], v[3]);
}

// x w for the scaled twiddle w = sigma (1 + i tau) (or i sigma (1 + i tau) when
// flagged), without the factor sigma: x (1 + i tau), then times i (forward) or
// -i (inverse, which uses conj(w)) where flagged
template <int DIR>
__device__ __forceinline__ cpx<double> scaled_input(cpx<double> x, double tau, bool rt) {
  const double t = DIR < 0 ? tau : -tau;
  const cpx<double> xt = {fma(-t, x.im, x.re), fma(t, x.re, x.im)};
  return {rt ? neg_if(xt.im, DIR < 0) : xt.re, rt ? neg_if(xt.re, DIR > 0) : xt.im};
}

// the radix-8 butterfly on the scaled record: the outputs of twiddle
// multiplication followed by dft8, with 66 FP64 operations instead of 80
template <int DIR>
__device__ __forceinline__ void radix8_scaled(cpx<double>* v, const Radix8Record* __restrict__ rec) {
  const double2* q = reinterpret_cast<const double2*>(rec);
  const double2 a0 = __ldg(q), a1 = __ldg(q + 1), a2 = __ldg(q + 2), a3 = __ldg(q + 3);
  const double2 a4 = __ldg(q + 4), a5 = __ldg(q + 5), a6 = __ldg(q + 6);
  const double s1h = __ldg(&rec->s1h);
  const long long rbits = __ldg(&rec->rot);
  const double tau[7] = {a0.x, a0.y, a1.x, a1.y, a2.x, a2.y, a3.x};
  const double s4 = a3.y, q62 = a4.x, s2 = a4.y, q51 = a5.x, q73 = a5.y, q31 = a6.x, s1 = a6.y;
  cpx<double> h[8];
  h[0] = v[0];
#pragma unroll
  for (int r = 1; r < 8; ++r) h[r] = scaled_input<DIR>(v[r], tau[r - 1], (rbits >> (r - 1)) & 1);
  // even inputs: x0 + sigma_4 h4, sigma_2 (h2 +- q62 h6)
  const cpx<double> s0 = {fma(s4, h[4].re, h[0].re), fma(s4, h[4].im, h[0].im)};
  const cpx<double> d0 = {fma(-s4, h[4].re, h[0].re), fma(-s4, h[4].im, h[0].im)};
  const cpx<double> u1 = {fma(q62, h[6].re, h[2].re), fma(q62, h[6].im, h[2].im)};
  const cpx<double> w1 = rot<DIR>(cpx<double>{fma(-q62, h[6].re, h[2].re), fma(-q62, h[6].im, h[2].im)});
  const cpx<double> e0 = {fma(s2, u1.re, s0.re), fma(s2, u1.im, s0.im)};
  const cpx<double> e2 = {fma(-s2, u1.re, s0.re), fma(-s2, u1.im, s0.im)};
  const cpx<double> e1 = {fma(s2, w1.re, d0.re), fma(s2, w1.im, d0.im)};
  const cpx<double> e3 = {fma(-s2, w1.re, d0.re), fma(-s2, w1.im, d0.im)};
  // odd inputs, on the common scale sigma_1
  const cpx<double> y0 = {fma(q51, h[5].re, h[1].re), fma(q51, h[5].im, h[1].im)};
  const cpx<double> z0 = {fma(-q51, h[5].re, h[1].re), fma(-q51, h[5].im, h[1].im)};
  const cpx<double> y1 = {fma(q73, h[7].re, h[3].re), fma(q73, h[7].im, h[3].im)};
  const cpx<double> z1 = rot<DIR>(cpx<double>{fma(-q73, h[7].re, h[3].re), fma(-q73, h[7].im, h[3].im)});
  const cpx<double> o0 = {fma(q31, y1.re, y0.re), fma(q31, y1.im, y0.im)};
  const cpx<double> o2 = {fma(-q31, y1.re, y0.re), fma(-q31, y1.im, y0.im)};
  const cpx<double> o1 = {fma(q31, z1.re, z0.re), fma(q31, z1.im, z0.im)};
  const cpx<double> o3 = {fma(-q31, z1.re, z0.re), fma(-q31, z1.im, z0.im)};
  // combine with W8^a (as in dft8), the scale sigma_1 inside the FMAs
  const double p1 = DIR < 0 ? o1.re + o1.im : o1.re - o1.im;
  const double r1 = DIR < 0 ? o1.im - o1.re : o1.im + o1.re;
  const double p3 = DIR < 0 ? o3.im - o3.re : o3.re + o3.im;
  const double r3 = DIR < 0 ? o3.re + o3.im : o3.re - o3.im;
  const double ha = DIR < 0 ? s1h : -s1h, hb = DIR < 0 ? -s1h : s1h;
  const cpx<double> t2 = rot<DIR>(o2);
  v[0] = {fma(s1, o0.re, e0.re), fma(s1, o0.im, e0.im)};
  v[4] = {fma(-s1, o0.re, e0.re), fma(-s1, o0.im, e0.im)};
  v[2] = {fma(s1, t2.re, e2.re), fma(s1, t2.im, e2.im)};
  v[6] = {fma(-s1, t2.re, e2.re), fma(-s1, t2.im, e2.im)};
  v[1] = {fma(s1h, p1, e1.re), fma(s1h, r1, e1.im)};
  v[5] = {fma(-s1h, p1, e1.re), fma(-s1h, r1, e1.im)};
  v[3] = {fma(ha, p3, e3.re), fma(hb, r3, e3.im)};
  v[7] = {fma(-ha, p3, e3.re), fma(-hb, r3, e3.im)};
}

template <int DIR>
__device__ __forceinline__ void radix4_scaled(cpx<double>* v, const Radix4Record* __restrict__ rec) {
  const double2* q = reinterpret_cast<const double2*>(rec);
  const double2 a0 = __ldg(q), a1 = __ldg(q + 1), a2 = __ldg(q + 2);
  const long long rbits = __ldg(&rec->rot);
  const double tau[3] = {a0.x, a0.y, a1.x};
  const double s2 = a1.y, q31 = a2.x, s1 = a2.y;
  cpx<double> h[4];
  h[0] = v[0];
#pragma unroll
  for (int r = 1; r < 4; ++r) h[r] = scaled_input<DIR>(v[r], tau[r - 1], (rbits >> (r - 1)) & 1);
  const cpx<double> s0 = {fma(s2, h[2].re, h[0].re), fma(s2, h[2].im, h[0].im)};
  const cpx<double> d0 = {fma(-s2, h[2].re, h[0].re), fma(-s2, h[2].im, h[0].im)};
  const cpx<double> u = {fma(q31, h[3].re, h[1].re), fma(q31, h[3].im, h[1].im)};
  const cpx<double> w = rot<DIR>(cpx<double>{fma(-q31, h[3].re, h[1].re), fma(-q31, h[3].im, h[1].im)});
  v[0] = {fma(s1, u.re, s0.re), fma(s1, u.im, s0.im)};
  v[2] = {fma(-s1, u.re, s0.re), fma(-s1, u.im, s0.im)};
  v[1] = {fma(s1, w.re, d0.re), fma(s1, w.im, d0.im)};
  v[3] = {fma(-s1, w.re, d0.re), fma(-s1, w.im, d0.im)};
}

template <int DIR>
__device__ __forceinline__ void radix3_scaled(cpx<double>* v, const Radix3Record* __restrict__ rec) {
  const double2* q = reinterpret_cast<const double2*>(rec);
  const double2 a0 = __ldg(q), a1 = __ldg(q + 1), a2 = __ldg(q + 2);
  const long long rbits = __ldg(&rec->rot);
  const double q21 = a1.x, s1 = a1.y, s1half = a2.x, ss1 = a2.y;
  const cpx<double> h1 = scaled_input<DIR>(v[1], a0.x, rbits & 1);
  const cpx<double> h2 = scaled_input<DIR>(v[2], a0.y, (rbits >> 1) & 1);
  const cpx<double> a = {fma(q21, h2.re, h1.re), fma(q21, h2.im, h1.im)};
  const cpx<double> b = {fma(-q21, h2.re, h1.re), fma(-q21, h2.im, h1.im)};
  const cpx<double> x0 = v[0];
  const cpx<double> t = {fma(-s1half, a.re, x0.re), fma(-s1half, a.im, x0.im)};
  v[0] = {fma(s1, a.re, x0.re), fma(s1, a.im, x0.im)};
  plus_minus_i<DIR>(t, ss1, b, v[1], v[2]);
}

template <int DIR>
__device__ __forceinline__ void radix2_scaled(cpx<double>* v, const Radix2Record* __restrict__ rec) {
  const double2 a0 = __ldg(reinterpret_cast<const double2*>(rec));
  const long long rbits = __ldg(&rec->rot);
  const cpx<double> h1 = scaled_input<DIR>(v[1], a0.x, rbits & 1);
  const double s1 = a0.y;
  const cpx<double> x0 = v[0];
  v[0] = {fma(s1, h1.re, x0.re), fma(s1, h1.im, x0.im)};
  v[1] = {fma(-s1, h1.re, x0.re), fma(-s1, h1.im, x0.im)};
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void fft_pass(cpx<T>* buf, int L, int nbatch, int Ns,
                                         const cpx<T>* __restrict__ stw, const cpx<T>* __restrict__ dtw,
                                         const FastDiv& dnb, const FastDiv& dns,
                                         const cpx<T>* __restrict__ gtw = nullptr) {
  constexpr int RP = (R + 1) & ~1;
  const int nb = L / R;
  const int total = nb * nbatch;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int batch = (int)fdiv((unsigned)b, dnb);
    const int j = b - batch * nb;
    const int g = (int)fdiv((unsigned)j, dns);
    const int k = j - g * Ns;
    cpx<T>* base = buf + batch * L + g * Ns * R + k;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[r * Ns];
    if constexpr (R <= 8 && R != 7 && std::is_same<T, double>::value) {
      if (gtw) {
        if constexpr (R == 5) radix5_scaled<DIR>(v, reinterpret_cast<const Radix5Record*>(gtw) + k);
        else if constexpr (R == 8) radix8_scaled<DIR>(v, reinterpret_cast<const Radix8Record*>(gtw) + k);
        else if constexpr (R == 4) radix4_scaled<DIR>(v, reinterpret_cast<const Radix4Record*>(gtw) + k);
        else if constexpr (R == 3) radix3_scaled<DIR>(v, reinterpret_cast<const Radix3Record*>(gtw) + k);
        else radix2_scaled<DIR>(v, reinterpret_cast<const Radix2Record*>(gtw) + k);
#pragma unroll
        for (int r = 0; r < R; ++r) base[r * Ns] = v[r];
        continue;
      }
    }
    if (Ns > 1) {
      const cpx<T>* tk = stw + k * RP;
      if constexpr (R <= 8) {
        cpx<T> w[R];
        load_stage_tw<R>(tk, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twmul<DIR>(v[r], w[r]);
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twmul<DIR>(v[r], ldg_c(tk + r));
      }
    }
    if constexpr (R <= 8) {
      dft_any<R, DIR>(v, dtw);
#pragma unroll
      for (int r = 0; r < R; ++r) base[r * Ns] = v[r];
    } else {
      // large odd prime: p_b = x_b + x_{R-b}, q_b = x_b - x_{R-b} in registers; each
      // output pair (a, R-a) is formed in a rolled loop over a and stored at once
      // (the butterfly's inputs are all in registers, so in-place is safe)
      constexpr int H = (R - 1) / 2;
      // p_b = x_b + x_{R-b} overwrites v[b], q_b = x_b - x_{R-b} overwrites v[R-b]
      cpx<T> y0 = v[0];
#pragma unroll
      for (int bb = 1; bb <= H; ++bb) {
        cpx<T> pb = v[bb] + v[R - bb];
        cpx<T> qb = v[bb] - v[R - bb];
        v[bb] = pb;
        v[R - bb] = qb;
        y0 = y0 + pb;
      }
      const cpx<T> x0 = v[0];
      base[0] = y0;
#pragma unroll 1
      for (int a = 1; a <= H; ++a) {
        cpx<T> A = x0, B = {(T)0, (T)0};
        int ab = 0;
#pragma unroll
        for (int bb = 1; bb <= H; ++bb) {
          ab += a;
          if (ab >= R) ab -= R;                  // ab = a * bb mod R
          cpx<T> w = ldg_c(dtw + ab);
          T c = w.re, sn = -w.im;                // w = exp(-2 pi i ab/R) = c - i sn
          A.re = fma(c, v[bb].re, A.re);
          A.im = fma(c, v[bb].im, A.im);
          B.re = fma(sn, v[R - bb].re, B.re);
          B.im = fma(sn, v[R - bb].im, B.im);
        }
        // y_a = A + DIR i B, y_{R-a} = A - DIR i B
        cpx<T> iB = DIR < 0 ? cpx<T>{B.im, -B.re} : cpx<T>{-B.im, B.re};
        base[a * Ns] = A + iB;
        base[(R - a) * Ns] = A - iB;
      }
    }
  }
  __syncthreads();
}

// Decimation in frequency: the transpose of the pass above.  Pass (R, Ns) as
// a matrix is (I (x) DFT_R (x) I_Ns) D with D the twiddles w^(r k); its transpose
// D (I (x) DFT_R (x) I_Ns) applies the R-point DFT first and the same twiddles
// after, on the same elements.  Since the DFT matrix is symmetric, running the
// transposed passes in reverse order on a sequence in natural order leaves
// the transform in digit-reversed order: output q at position perm[q], the
// position the DIT load gives input q.  Plain twiddle tables only (the FP32 and
// double-float kernels).
template <int R, int DIR, typename T>
__device__ __forceinline__ void fft_pass_dif(cpx<T>* buf, int L, int nbatch, int Ns,
                                             const cpx<T>* __restrict__ stw, const cpx<T>* __restrict__ dtw,
                                             const FastDiv& dnb, const FastDiv& dns) {
  constexpr int RP = (R + 1) & ~1;
  const int nb = L / R;
  const int total = nb * nbatch;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int batch = (int)fdiv((unsigned)b, dnb);
    const int j = b - batch * nb;
    const int g = (int)fdiv((unsigned)j, dns);
    const int k = j - g * Ns;
    cpx<T>* base = buf + batch * L + g * Ns * R + k;
    const cpx<T>* tk = stw + k * RP;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[r * Ns];
    if constexpr (R <= 8) {
      dft_any<R, DIR>(v, dtw);
      if (Ns > 1) {
        cpx<T> w[R];
        load_stage_tw<R>(tk, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = out_norm<T>(twmul<DIR>(v[r], w[r]));
      }
#pragma unroll
      for (int r = 0; r < R; ++r) base[r * Ns] = v[r];
    } else {
      // large odd prime: as in fft_pass, each output pair (a, R - a) formed in a
      // rolled loop, then multiplied by its twiddle and stored
      constexpr int H = (R - 1) / 2;
      cpx<T> y0 = v[0];
#pragma unroll
      for (int bb = 1; bb <= H; ++bb) {
        cpx<T> pb = v[bb] + v[R - bb];
        cpx<T> qb = v[bb] - v[R - bb];
        v[bb] = pb;
        v[R - bb] = qb;
        y0 = y0 + pb;
      }
      const cpx<T> x0 = v[0];
      base[0] = y0;
#pragma unroll 1
      for (int a = 1; a <= H; ++a) {
        cpx<T> A = x0, B = {(T)0, (T)0};
        int ab = 0;
#pragma unroll
        for (int bb = 1; bb <= H; ++bb) {
          ab += a;
          if (ab >= R) ab -= R;
          cpx<T> w = ldg_c(dtw + ab);
          T c = w.re, sn = -w.im;
          A.re = fma(c, v[bb].re, A.re);
          A.im = fma(c, v[bb].im, A.im);
          B.re = fma(sn, v[R - bb].re, B.re);
          B.im = fma(sn, v[R - bb].im, B.im);
        }
        cpx<T> iB = DIR < 0 ? cpx<T>{B.im, -B.re} : cpx<T>{-B.im, B.re};
        cpx<T> ya = A + iB, yb = A - iB;
        if (Ns > 1) {
          ya = out_norm<T>(twmul<DIR>(ya, ldg_c(tk + a)));
          yb = out_norm<T>(twmul<DIR>(yb, ldg_c(tk + (R - a))));
        }
        base[a * Ns] = ya;
        base[(R - a) * Ns] = yb;
      }
    }
  }
  __syncthreads();
}

// Full decimation-in-frequency transform: natural order in, output q at
// position perm[q] (perm as for fft_run's input).  Expects a barrier before entry.
template <int DIR, bool BIG, typename T>
__device__ __forceinline__ void fft_run_dif(cpx<T>* buf, int nbatch, const FftDesc& d, const cpx<T>* __restrict__ tw) {
  int Ns = d.L;
  for (int s = d.nstages - 1; s >= 0; --s) {
    const int R = d.radix[s];
    Ns /= R;                                   // R_1 ... R_{s-1}
    const cpx<T>* stw = tw + d.tw_off[s];
    const cpx<T>* dtw = tw + d.dft_off[s];
    switch (R) {
      case 2: fft_pass_dif<2, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 3: fft_pass_dif<3, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 4: fft_pass_dif<4, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 5: fft_pass_dif<5, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 7: fft_pass_dif<7, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 8: fft_pass_dif<8, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      default: break;
    }
    if constexpr (BIG) {
      switch (R) {
      case 11: fft_pass_dif<11, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 13: fft_pass_dif<13, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 17: fft_pass_dif<17, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 19: fft_pass_dif<19, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 23: fft_pass_dif<23, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 29: fft_pass_dif<29, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 31: fft_pass_dif<31, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      default: break;
      }
    }
  }
}

// Full transform of sequences stored in digit-reversed order (position
// perm[q] holds input q; see the host's digit_reversal): DIR = -1 computes
// sum_q a_q exp(-2 pi i q k / L) (unnormalised), DIR = +1 the same with exp(+...),
// leaving the result in natural order.  Expects a barrier before entry.
// BIG = false: radices 2, 3, 4, 5, 7, 8 only (keeps register allocation tight);
// BIG = true adds the odd primes 11 .. 31 for lengths that need them.
template <int DIR, bool BIG, typename T>
__device__ __forceinline__ void fft_run(cpx<T>* buf, int nbatch, const FftDesc& d, const cpx<T>* __restrict__ tw) {
  int Ns = 1;
  for (int s = 0; s < d.nstages; ++s) {
    const int R = d.radix[s];
    const cpx<T>* stw = tw + d.tw_off[s];
    const cpx<T>* dtw = tw + d.dft_off[s];
    // the scaled radix-5 records serve the FP64 kernels only
    const cpx<T>* gtw = (std::is_same<T, double>::value && d.g_off[s] >= 0) ? tw + d.g_off[s] : nullptr;
    switch (R) {
      case 2: fft_pass<2, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s], gtw); break;
      case 3: fft_pass<3, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s], gtw); break;
      case 4: fft_pass<4, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s], gtw); break;
      case 5: fft_pass<5, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s], gtw); break;
      case 7: fft_pass<7, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 8: fft_pass<8, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s], gtw); break;
      default: break;
    }
    if constexpr (BIG) {
      switch (R) {
      case 11: fft_pass<11, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 13: fft_pass<13, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 17: fft_pass<17, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 19: fft_pass<19, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 23: fft_pass<23, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 29: fft_pass<29, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      case 31: fft_pass<31, DIR>(buf, d.L, nbatch, Ns, stw, dtw, d.div_nb[s], d.div_ns[s]); break;
      default: break;  // the host never builds other radices
      }
    }
    Ns *= R;
  }
}

}  // namespace sp
