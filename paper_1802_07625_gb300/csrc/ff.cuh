// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, which carries about 48 significant bits. Sums use the error-free
// two-sum of two floats (Knuth), products the error-free product by fused multiply-add;
// each result is renormalised. Used for the mixed path's compensated second transform pass,
// where FP32 rounding at the scale of a line's largest values would swamp densities far
// below it.
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
// the operands, which is the bound a transform's error analysis uses (a sum that cancels
// keeps the absolute error of its operands).
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // p + e = a.hi * b.hi exactly
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - b * ff(q1, 0.0f);
  const float q2 = __fdiv_rn(__fadd_rn(r.hi, r.lo), b.hi);
  return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

struct ff2 {
  ff x, y;
};
template <> struct vec2<ff> { using type = ff2; };

}  // namespace cg
