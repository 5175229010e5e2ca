// f32x2.cuh -- packed pairs of FP32 numbers and the double-float operations
// built on them.
//
// Blackwell executes add / sub / mul / fma on a pair of FP32 lanes held in one
// 64-bit register (PTX `.f32x2`, sm_100 and later) with one issued
// instruction.  The FP32 pipe does the same lane work as for two scalar
// instructions, but the pair takes one issue slot instead of two, which is
// what bounds double-float code (about a dozen dependent FP32 operations per
// multiply-add).  Each lane is rounded to nearest exactly as the scalar
// instruction is, so the error-free transformations of df64.cuh stay exact
// lane by lane and the packed results equal the scalar ones bit for bit.
//
// The asm statements are not volatile: they are pure functions of their
// inputs, which leaves the compiler free to schedule them.
#pragma once

#include <cuda_runtime.h>

namespace bsm {

typedef unsigned long long f32x2;  // (lane 0, lane 1)

__device__ __forceinline__ f32x2 pk2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(f32x2 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f32x2 swap2(f32x2 x) {
  float a, b;
  up2(x, a, b);
  return pk2(b, a);
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Two double-float values, one per lane.
//  dfp2:  hi parts and lo parts;
//  dfn2:  hi parts and the NEGATED lo parts (the form a product chain
//         produces for free, see prod2);
//  dfv2:  an operand with its negation (hi, lo, -hi, -lo), so that the exact
//         error of a product is an fma with a positive coefficient.
struct dfp2 {
  f32x2 hi, lo;
};
struct dfn2 {
  f32x2 hi, nlo;
};
struct dfv2 {
  f32x2 hi, lo, nhi, nlo;
};

// c = a * b for a coefficient a broadcast to both lanes (ah, al) and a pair
// b: the rounded product of the high parts and, negated, its exact error
// (Dekker's product through an fma) plus the two cross terms -- the same
// operations as df64.cuh's product, lane by lane.
__device__ __forceinline__ dfn2 prod2(f32x2 ah, f32x2 al, const dfv2& b) {
  dfn2 r;
  r.hi = mul2(ah, b.hi);
  f32x2 ne = fma2(ah, b.nhi, r.hi);  // p - a.hi b.hi = -(exact error of p)
  ne = fma2(ah, b.nlo, ne);
  r.nlo = fma2(al, b.nhi, ne);
  return r;
}

// c += a * b: the product as in prod2, Knuth's TwoSum of the high parts into
// the accumulator, low parts added in FP32 (df64.cuh's fma, lane by lane)
__device__ __forceinline__ void fmacc2(f32x2 ah, f32x2 al, const dfv2& b, dfn2& c) {
  const f32x2 p = mul2(ah, b.hi);
  f32x2 ne = fma2(ah, b.nhi, p);
  ne = fma2(ah, b.nlo, ne);
  ne = fma2(al, b.nhi, ne);
  const f32x2 s = add2(c.hi, p);
  const f32x2 bb = sub2(s, c.hi);
  const f32x2 e = add2(sub2(c.hi, sub2(s, bb)), sub2(p, bb));
  c.hi = s;
  c.nlo = sub2(add2(c.nlo, ne), e);
}

// x += y with y given as (hi, negated lo): TwoSum of the high parts, low
// parts added in FP32 (df64.cuh's sum, lane by lane)
__device__ __forceinline__ void padd(dfp2& x, f32x2 yh, f32x2 ynlo) {
  const f32x2 s = add2(x.hi, yh);
  const f32x2 bb = sub2(s, x.hi);
  const f32x2 e = add2(sub2(x.hi, sub2(s, bb)), sub2(yh, bb));
  x.hi = s;
  x.lo = add2(e, sub2(x.lo, ynlo));
}

}  // namespace bsm
