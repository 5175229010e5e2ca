// df64.cuh -- double-float ("DF64") arithmetic: a real number carried as an
// unevaluated sum hi + lo of two FP32 numbers, about 48 significand bits.
//
// GB300 executes FP32 about 60 times faster than FP64 (73 vs 1.2 TFLOP/s
// measured), so an FP64-accurate hop is cheaper in FP32 pairs than in FP64.
// The building blocks are the classical error-free transformations:
//   two_sum   Knuth, TAOCP vol. 2, Sec. 4.2.2 (TwoSum): s + e = a + b exactly;
//   two_prod  Dekker 1971 with a fused multiply-add: p + e = a * b exactly;
// and the double-word sum and product built from them (Dekker 1971; the
// error bounds are analysed in Joldes, Muller, Popescu, ACM TOMS 2017).
// Results of df_add / df_fma are left unnormalised (|lo| may reach a few
// ulp(hi)); df_norm (fast two-sum) renormalises before a value is stored.
// Every operation uses the explicitly rounded intrinsics, so the compiler
// cannot contract a product into a following sum and break the
// transformations.
#pragma once

#include <cuda_runtime.h>

namespace bsm {

// the df overload of fma below must not hide the standard float/double ones
using ::fma;

struct df {
  float hi, lo;
  __host__ __device__ df() {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // exact split of a double into hi + lo (lo is the rounded remainder)
  __device__ __forceinline__ explicit df(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ __forceinline__ explicit df(int x) : hi((float)x), lo(0.f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (6 flops, no ordering condition)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}

// s + e = a + b exactly when |a| >= |b| (3 flops)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df df_norm(df x) { return fast_two_sum(x.hi, x.lo); }

__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }

// x + y (unnormalised)
__device__ __forceinline__ df operator+(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return s;
}
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df& operator+=(df& x, df y) { return x = x + y; }

// x * y: exact product of the high parts plus the two cross terms
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// c + a * b (unnormalised): two_prod of the high parts, the cross terms in
// FP32, and a two_sum into the accumulator
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df s = two_sum(c.hi, p);
  s.lo = __fadd_rn(s.lo, __fadd_rn(c.lo, e));
  return s;
}

}  // namespace bsm
