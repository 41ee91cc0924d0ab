// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers, which
// carries about 48 significant bits. Sums use the error-free two-sum of the high parts
// (Knuth) and add the low parts in FP32; products take the error-free product of the high
// parts by fused multiply-add plus the two cross terms. Results are not renormalised: lo
// may exceed ulp(hi)/2 by a small factor, and after a cancellation of the high parts it may
// hold most of the value, which is then tiny against the operands. Every error stays within
// a small multiple of 2^-44 of the operands' magnitudes, the bound a transform's error
// analysis uses. Used for the mixed path's compensated second transform pass, where FP32
// rounding at the scale of a line's largest values would swamp densities far below it.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace cg {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest float-float to d: the float nearest d and the float nearest the remainder
  // (constexpr: the transform's constant twiddles fold at compile time)
  __host__ __device__ constexpr ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  // integers below 2^24 are exact floats
  __host__ __device__ constexpr ff(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ constexpr ff(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}
// the same when |a| >= |b|
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// The sum's error is within a small multiple of 2^-44 (|a| + |b|): relative to the size of
// the operands (a sum that cancels keeps the absolute error of its operands).
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
// The product drops a.lo * b.lo, which is below 2^-44 |a| |b| while the low parts are small;
// where a cancellation left a low part as large as its high part, the value is itself below
// 2^-22 of the operands that formed it, and the dropped term is as small in absolute terms.
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // p + e = a.hi * b.hi exactly
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff(p, e);
}
__device__ __forceinline__ ff operator/(ff a, ff b) {
  b = ff_two_sum(b.hi, b.lo);  // normalised divisor: q2 below divides by b.hi alone
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - b * ff(q1, 0.0f);
  const float q2 = __fdiv_rn(__fadd_rn(r.hi, r.lo), b.hi);
  return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
// by the sign of the difference (the parts of an unnormalised value do not order it)
__device__ __forceinline__ bool operator>(ff a, ff b) {
  const ff d = a - b;
  return __fadd_rn(d.hi, d.lo) > 0.0f;
}

struct ff2 {
  ff x, y;
};
template <> struct vec2<ff> { using type = ff2; };

}  // namespace cg
