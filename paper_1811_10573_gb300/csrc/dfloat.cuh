// Double-float arithmetic (hi + lo, two floats, 48-bit significand) from the
// classical error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker),
// TwoProd via FMA, and the double-word addition and multiplication built on
// them (Joldes, Muller and Popescu; accurate variants, relative error a few
// units of 2^-48).  Rounding-sensitive steps use __f*_rn intrinsics so the
// compiler cannot contract or reassociate them.  Shared by the double-float
// normal-equation kernels of the contexts and of the batch.
#pragma once

#include <cuda_runtime.h>

namespace cpals {
namespace dfa {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {   // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  const dfl t = two_sum(x.lo, y.lo);
  const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const dfl c = two_prod(x.hi, y.hi);
  const float t0 = __fmul_rn(x.lo, y.lo);
  const float t1 = __fmaf_rn(x.hi, y.lo, t0);
  const float t2 = __fmaf_rn(x.lo, y.hi, t1);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, t2));
}
// "sloppy" double-word addition (one TwoSum): error bounded relative to
// |x| + |y| (a few units of 2^-48); used where that backward-error bound is
// what matters (the Cholesky trailing update)
__device__ __forceinline__ dfl df_add_fast(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// 1/sqrt(a): float reciprocal square root refined by one Newton step,
// r = r0 + r0 (1 - a r0^2) / 2.  The residual is formed with FMAs:
// a.hi r0 = h + dh exactly, 1 - h r0 is exact before its one rounding (it is
// ~2^-22), then the small terms dh r0 and a.lo r0^2 are taken off.
__device__ __forceinline__ dfl df_rsqrt(dfl a) {
  const float r0 = rsqrtf(a.hi);
  const float h = __fmul_rn(a.hi, r0);
  const float dh = __fmaf_rn(a.hi, r0, -h);
  const float r02 = __fmul_rn(r0, r0);
  float e = __fmaf_rn(-h, r0, 1.f);
  e = __fmaf_rn(-dh, r0, e);
  e = __fmaf_rn(-a.lo, r02, e);
  return fast_two_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), e));
}
__device__ __forceinline__ dfl df_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_dbl(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float2 pk(dfl a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ dfl upk(float2 a) { return {a.x, a.y}; }


}  // namespace dfa
}  // namespace cpals
