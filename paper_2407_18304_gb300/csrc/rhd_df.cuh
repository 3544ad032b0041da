// rhd_df.cuh -- float-float ("double-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  GB300 issues FP64 at 1/64 of its FP32 rate, so a
// float-float operation (5 to 20 FP32 instructions) costs a fraction of one
// FP64 instruction.  The building blocks are the error-free transformations of
// Knuth (two-sum) and Dekker (fast two-sum), and the product error by a fused
// multiply-add; the compound operations follow the "sloppy" double-double
// forms of Hida, Li & Bailey (2001), whose error is a few units of 2^-48 of the
// operands' size (not of the result's): what a residual evaluation needs, whose
// accuracy is judged against the size of the terms that cancel in it.
//
// The intrinsics __fadd_rn / __fmul_rn / __fsub_rn keep the compiler from
// contracting the transformations' products and sums into FMAs.
#pragma once
#include <cuda_runtime.h>

namespace rhd {

struct dflt {
  float hi, lo;
};

__device__ __forceinline__ dflt df_from_float(float a) { return dflt{a, 0.0f}; }

// Exponent of an FP32 subnormal's bit pattern b (0 < b < 2^23): x = b 2^-149.
__device__ __forceinline__ int df_exponent_sub(int b) { return (32 - __clz(b)) - 149; }

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ dflt two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dflt{s, e};
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker).
__device__ __forceinline__ dflt fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dflt{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a b exactly (barring underflow).
__device__ __forceinline__ dflt two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dflt{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dflt operator-(dflt a) { return dflt{-a.hi, -a.lo}; }

__device__ __forceinline__ dflt operator+(dflt a, dflt b) {
  const dflt s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dflt operator-(dflt a, dflt b) { return a + (-b); }
__device__ __forceinline__ dflt operator+(dflt a, float b) {
  const dflt s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ dflt operator-(dflt a, float b) { return a + (-b); }
__device__ __forceinline__ dflt operator+(float a, dflt b) { return b + a; }
__device__ __forceinline__ dflt operator-(float a, dflt b) { return (-b) + a; }

__device__ __forceinline__ dflt operator*(dflt a, dflt b) {
  const dflt p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ dflt operator*(dflt a, float b) {
  const dflt p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ dflt operator*(float a, dflt b) { return b * a; }

// Multiplication by a power of two (exact).
__device__ __forceinline__ dflt df_scale(dflt a, float p2) { return dflt{a.hi * p2, a.lo * p2}; }

// a / b: a first quotient from the FP32 reciprocal, then one correction from
// the remainder a - q1 b, formed with an exact product.
__device__ __forceinline__ dflt operator/(dflt a, dflt b) {
  const float r = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, r);
  const dflt p = two_prod(q1, b.hi);
  const float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), fmaf(-q1, b.lo, a.lo));
  return fast_two_sum(q1, __fmul_rn(rem, r));
}

// 1 / b.
__device__ __forceinline__ dflt df_rcp(dflt b) {
  const float r = __frcp_rn(b.hi);
  const dflt p = two_prod(r, b.hi);
  const float rem = __fsub_rn(__fsub_rn(1.0f - p.hi, p.lo), __fmul_rn(r, b.lo));
  return fast_two_sum(r, __fmul_rn(rem, r));
}

// sqrt(a), a >= 0: s from the FP32 square root, then s + (a - s^2) / (2 s).
__device__ __forceinline__ dflt df_sqrt(dflt a) {
  if (!(a.hi > 0.0f)) return dflt{0.0f, 0.0f};
  const float s = __fsqrt_rn(a.hi);
  const dflt p = two_prod(s, s);
  const float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
  return fast_two_sum(s, __fmul_rn(rem, __fdividef(0.5f, s)));
}

// The binary exponent e of a nonzero float, x = m 2^e with m in [0.5, 1)
// (FP32 subnormals included), from the bit pattern.
__device__ __forceinline__ int df_exponent(float x) {
  int b = __float_as_int(x) & 0x7FFFFFFF;
  if (b < 0x00800000) return df_exponent_sub(b);
  return (b >> 23) - 126;
}

// a / b with both first scaled by the same power of two, so that b is of
// order one: the quotient of two tiny (or huge) values, whose FP32 reciprocal
// would overflow (or underflow), stays exact to float-float accuracy.  b != 0.
__device__ __forceinline__ dflt df_div_scaled(dflt a, dflt b) {
  const int e = df_exponent(b.hi);
  const int e1 = e / 2, e2 = e - e1;  // two normal powers of two: e in [-149, 128]
  const float s1 = __int_as_float((127 - e1) << 23), s2 = __int_as_float((127 - e2) << 23);
  return df_scale(df_scale(a, s1), s2) / df_scale(df_scale(b, s1), s2);
}

// Order by value (hi first; lo breaks ties).
__device__ __forceinline__ bool operator<(dflt a, dflt b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(dflt a, dflt b) { return b < a; }
__device__ __forceinline__ bool df_pos(dflt a) { return a.hi > 0.0f; }
__device__ __forceinline__ dflt df_min(dflt a, dflt b) { return b < a ? b : a; }
__device__ __forceinline__ dflt df_max(dflt a, dflt b) { return a < b ? b : a; }

// A double times 2^-sh as a float-float, from the bit pattern: the first 24
// significant bits cut (not rounded) into hi, the next 24 into lo.  No FP64
// instruction; results below FP32's normal range give 0, above it +-inf.
__device__ __forceinline__ float df_cut_bits(int hw, int lw, int sh) {
  const int E = (hw >> 20) & 0x7FF;
  const unsigned sign = (unsigned)hw & 0x80000000u;
  if (E == 0) return __int_as_float((int)sign);
  const int fe = E - 1023 - sh + 127;
  if (fe <= 0) return __int_as_float((int)sign);
  if (fe >= 255) return __int_as_float((int)(sign | 0x7F800000u));
  const unsigned frac = ((unsigned)(hw & 0xFFFFF) << 3) | ((unsigned)lw >> 29);
  return __int_as_float((int)(sign | ((unsigned)fe << 23) | frac));
}

// The part of a normal double below its first 24 significant bits (the low
// 29 bits of its fraction, r 2^(E - 1075)) times 2^-sh, cut to 24 bits, from
// the bit pattern alone: the exact x - (its 24-bit cut) that an FP64
// subtraction would form, then cut as df_cut_bits cuts.  Integer instructions
// only; results below FP32's normal range give 0.
__device__ __forceinline__ float df_rest_bits(int hw, int lw, int sh) {
  const int E = (hw >> 20) & 0x7FF;
  const unsigned sign = (unsigned)hw & 0x80000000u;
  const unsigned r = (unsigned)lw & 0x1FFFFFFFu;
  if (r == 0u) return 0.0f;  // an exact cut: the FP64 difference would be +0
  if (E == 0) return __int_as_float((int)sign);
  const int top = 31 - __clz((int)r);  // the leading one of r: r in [2^top, 2^(top+1))
  const int fe = top + E - 1075 - sh + 127;
  if (fe <= 0) return __int_as_float((int)sign);
  if (fe >= 255) return __int_as_float((int)(sign | 0x7F800000u));
  const unsigned m = (top >= 23 ? (r >> (top - 23)) : (r << (23 - top))) & 0x7FFFFFu;
  return __int_as_float((int)(sign | ((unsigned)fe << 23) | m));
}

__device__ __forceinline__ dflt df_from_double(double x, int sh) {
  const int hw = __double2hiint(x), lw = __double2loint(x);
  return dflt{df_cut_bits(hw, lw, sh), df_rest_bits(hw, lw, sh)};
}

}  // namespace rhd
