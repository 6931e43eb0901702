// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two IEEE single-precision numbers with |lo| <= ulp(hi)/2, about 48 bits of
// significand.  On this GPU the FP32 pipes issue 69x faster than the FP64
// pipe, so transforms written in df64 reach FP64-level accuracy faster than
// native double arithmetic.
//
// The operations are the classical error-free transformations: Knuth's TwoSum
// (a + b = s + e exactly), Dekker/Kahan's FastTwoSum for renormalisation, and
// the FMA-based TwoProduct (a b = p + e exactly, e = fma(a, b, -p)); additions
// use the "sloppy" double-double sum (Bailey's QD library design), whose error
// is bounded relative to |a| + |b|, the norm-wise bound an FFT error analysis
// needs.  Every float operation goes through __f*_rn intrinsics so the compiler
// cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace sp {

using ::fma;  // keep the float / double overloads visible next to the double-float one

struct alignas(8) dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // split of a double constant (exact to ~2^-48 relative)
  __host__ __device__ constexpr explicit dd(double x)
      : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
  __host__ __device__ constexpr explicit dd(int x) : dd(static_cast<double>(x)) {}
};

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float hi = __fadd_rn(s, e);
  float lo = __fsub_rn(e, __fsub_rn(hi, s));
  return {hi, lo};
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float hi = __fadd_rn(p, e);
  float lo = __fsub_rn(e, __fsub_rn(hi, p));
  return {hi, lo};
}

// a * b + c with one renormalisation of the product folded into the sum
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  // (p + e) + c: TwoSum of the leading parts, then the tails
  float s = __fadd_rn(p, c.hi);
  float bb = __fsub_rn(s, p);
  float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  float hi = __fadd_rn(s, t);
  float lo = __fsub_rn(t, __fsub_rn(hi, s));
  return {hi, lo};
}

// Unnormalised forms for values that feed further double-float operations
// inside one butterfly: the same operations without the final renormalisation
// (FastTwoSum, three operations), returning (hi, lo) with hi + lo the same
// value and |lo| a few ulp(hi) instead of at most half of one.  TwoSum and the
// FMA TwoProduct are exact for any float inputs, so the next operation loses
// nothing but the last bit or two of the lo parts' FP32 sum; stored results go
// through dd_norm.
__device__ __forceinline__ dd dd_norm(dd a) {
  float hi = __fadd_rn(a.hi, a.lo);
  float lo = __fsub_rn(a.lo, __fsub_rn(hi, a.hi));
  return {hi, lo};
}
__device__ __forceinline__ dd dd_add_u(dd a, dd b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ dd dd_sub_u(dd a, dd b) { return dd_add_u(a, dd(-b.hi, -b.lo)); }
__device__ __forceinline__ dd dd_mul_u(dd a, dd b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}
__device__ __forceinline__ dd dd_fma_u(dd a, dd b, dd c) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s = __fadd_rn(p, c.hi);
  float bb = __fsub_rn(s, p);
  float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  return {s, __fadd_rn(t, __fadd_rn(e, c.lo))};
}

__device__ __forceinline__ dd operator+(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return dd_sub(a, b); }
__device__ __forceinline__ dd operator-(dd a) { return dd_neg(a); }
__device__ __forceinline__ dd operator*(dd a, dd b) { return dd_mul(a, b); }
__device__ __forceinline__ dd fma(dd a, dd b, dd c) { return dd_fma(a, b, c); }

// double <-> df64 conversions (two F2F and one DADD per value)
__device__ __forceinline__ dd dd_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

}  // namespace sp
